// Compile-time Stockham plane kernels for the further sizes 60, 72, 75, 80, double-float (see
// plane_fast_impl.cuh).
#include "plane_fast_impl.cuh"

namespace wdf {

using MoreDfB = PlaneFastSizes<df64, 60, 72, 75, 80>;

bool launch_plane_more_df_b(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st) {
  return MoreDfB::launch(f, op, nblk, pa, st);
}
void set_plane_more_limits_df_b(const Geo &g) { MoreDfB::limits(g); }

}  // namespace wdf

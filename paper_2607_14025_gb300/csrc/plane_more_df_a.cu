// Compile-time Stockham plane kernels for the further sizes 36, 40, 45, 50, 54, double-float (see
// plane_fast_impl.cuh).
#include "plane_fast_impl.cuh"

namespace wdf {

using MoreDfA = PlaneFastSizes<df64, 36, 40, 45, 50, 54>;

bool launch_plane_more_df_a(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st) {
  return MoreDfA::launch(f, op, nblk, pa, st);
}
void set_plane_more_limits_df_a(const Geo &g) { MoreDfA::limits(g); }

}  // namespace wdf

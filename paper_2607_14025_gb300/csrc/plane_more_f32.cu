// Compile-time Stockham plane kernels for the further sizes, float (see plane_fast_impl.cuh).
#include "plane_fast_impl.cuh"

namespace wdf {

using MoreF32 = PlaneFastSizes<float, 36, 40, 45, 50, 54, 60, 72, 75, 80>;

bool launch_plane_more_f32(const FftCtx<float> &f, int op, int nblk, const PlaneArgs<float> &pa, cudaStream_t st) {
  return MoreF32::launch(f, op, nblk, pa, st);
}
void set_plane_more_limits_f32(const Geo &g) { MoreF32::limits(g); }

}  // namespace wdf

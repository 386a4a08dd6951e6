// Batched Gamma-point 3-D FFTs between the plane-wave sphere and the real-space grid.
//
// Data model (built on the host, see layout.cu):
//  * A real function f is stored by "rep columns": for each (n1, n2) with n1 > 0, or n1 = 0 and
//    n2 > 0, plus the column (0, 0), the coefficients f(n1, n2, n3) for every n3 of the sphere in
//    that column. The mirror column (-n1, -n2) follows from f(-G) = conj(f(G)). Column (0, 0) is
//    stored in full (both signs of n3). Inner products weight column (0, 0) by 1, others by 2.
//  * Two real functions a, b travel together as one complex function F = a + i b (Gamma pairing):
//    one complex FFT serves two real transforms.
//  * Column buffer cb[pair][z][j]: after the n3 transforms, the value of F at grid plane z for disk
//    column j (j < K: rep column j; j >= K: mirror of rep column j - K + 1).
//
// G -> r: k_zpass_g2r (n3 transforms of the disk columns) then a plane kernel (n2 transforms of
// the occupied n1 columns, n1 transforms of all rows). r -> G runs the same steps backwards.
// Plane kernels hold one z plane of one pair in shared memory and fuse the pointwise work.
#include "fft.cuh"
#include "kernels.cuh"
#include "zpass.cuh"

namespace wdf {

// ---------------------------------------------------------------------------------------------
// plane kernels (one z plane of one pair per block)

template <typename T>
__device__ void plane_g2r(cplx<T> *tile, const cplx<T> *__restrict__ cbz, const Geo &g, const Plan1D &P1,
                          const Plan1D &P2, const cplx<T> *tw1, const cplx<T> *tw2, const int *xact) {
  const int npt = g.n2 * g.pitch;
  for (int i = threadIdx.x; i < npt; i += blockDim.x) tile[i] = mkc<T>(0, 0);
  __syncthreads();
  for (int j = threadIdx.x; j < g.ndisk; j += blockDim.x) tile[g.tile_idx[j]] = cbz[j];
  __syncthreads();
  fft_lines<T, true>(tile, g.nxact, xact, 0, g.pitch, P2, tw2);  // along n2, occupied n1 columns
  fft_lines<T, true>(tile, g.n2, nullptr, g.pitch, 1, P1, tw1);  // along n1, every row
}

template <typename T>
__device__ void plane_r2g(cplx<T> *tile, cplx<T> *__restrict__ cbz, const Geo &g, const Plan1D &P1,
                          const Plan1D &P2, const cplx<T> *tw1, const cplx<T> *tw2, const int *xact) {
  fft_lines<T, false>(tile, g.n2, nullptr, g.pitch, 1, P1, tw1);
  fft_lines<T, false>(tile, g.nxact, xact, 0, g.pitch, P2, tw2);
  for (int j = threadIdx.x; j < g.ndisk; j += blockDim.x) cbz[j] = tile[g.tile_idx[j]];
}

template <typename T>
__device__ void plane_setup(cplx<T> *&tile, cplx<T> *&tw1, cplx<T> *&tw2, int *&xact, const Geo &g,
                            const cplx<T> *tw1g, const cplx<T> *tw2g) {
  extern __shared__ __align__(16) unsigned char smraw[];
  tw1 = reinterpret_cast<cplx<T> *>(smraw);
  tw2 = tw1 + kMaxN;
  tile = tw2 + kMaxN;
  xact = reinterpret_cast<int *>(tile + g.n2 * g.pitch);
  for (int i = threadIdx.x; i < g.n1; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < g.n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < g.nxact; i += blockDim.x) xact[i] = g.xact[i];
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) k_plane(Geo g, Plan1D P1, Plan1D P2, const cplx<T> *__restrict__ tw1g,
                                                     const cplx<T> *__restrict__ tw2g, PlaneArgs<T> pa) {
  cplx<T> *tile, *tw1, *tw2;
  int *xact;
  plane_setup<T>(tile, tw1, tw2, xact, g, tw1g, tw2g);
  const int z = blockIdx.y;
  const size_t plane = (size_t)g.n1 * g.n2;
  const size_t cbpair = (size_t)g.n3 * g.ldcb;
  if (OP == OP_VLOC) {
    const int q = blockIdx.x;
    cplx<T> *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    plane_g2r<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
    const T *v = pa.field + (size_t)z * plane;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
      const int y = i / g.n1, x = i - y * g.n1;
      tile[y * g.pitch + x] = cscal<T>(tile[y * g.pitch + x], v[i]);
    }
    __syncthreads();
    plane_r2g<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
  } else if (OP == OP_G2R) {
    const int q = blockIdx.x;
    const cplx<T> *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    plane_g2r<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
    cplx<T> *out = pa.grid + (size_t)q * g.n3 * plane + (size_t)z * plane;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
      const int y = i / g.n1, x = i - y * g.n1;
      out[i] = tile[y * g.pitch + x];
    }
  } else if (OP == OP_PROD_R2G) {
    // pair q = pp * nocc + v:  F(r) = psi_v(r) * (dV_2pp + i dV_2pp+1)(r)
    const int q = blockIdx.x;
    const int v = q % pa.nocc, pp = q / pa.nocc;
    const T *psi = pa.field + (size_t)v * g.n3 * plane + (size_t)z * plane;
    const cplx<T> *dv = pa.grid + (size_t)pp * g.n3 * plane + (size_t)z * plane;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
      const int y = i / g.n1, x = i - y * g.n1;
      tile[y * g.pitch + x] = cscal<T>(dv[i], psi[i]);
    }
    __syncthreads();
    cplx<T> *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    plane_r2g<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
  } else {  // OP_ACCUM: acc(r) = sum_v psi_v(r) G2R(cb[pp * nocc + v]); then r -> G into cb2[pp]
    const int pp = blockIdx.x;
    cplx<T> *acc = pa.grid + (size_t)pp * g.n3 * plane + (size_t)z * plane;
    for (int v = 0; v < pa.nocc; ++v) {
      const cplx<T> *cbz = pa.cb + ((size_t)pp * pa.nocc + v) * cbpair + (size_t)z * g.ldcb;
      plane_g2r<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
      const T *psi = pa.field + (size_t)v * g.n3 * plane + (size_t)z * plane;
      for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
        const int y = i / g.n1, x = i - y * g.n1;
        const cplx<T> t = cscal<T>(tile[y * g.pitch + x], psi[i]);
        acc[i] = (v == 0) ? t : cadd<T>(acc[i], t);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
      const int y = i / g.n1, x = i - y * g.n1;
      tile[y * g.pitch + x] = acc[i];
    }
    __syncthreads();
    cplx<T> *cbz = pa.cb2 + (size_t)pp * cbpair + (size_t)z * g.ldcb;
    plane_r2g<T>(tile, cbz, g, P1, P2, tw1, tw2, xact);
  }
}

// ---------------------------------------------------------------------------------------------
// host launchers

template <typename T> size_t zpass_smem(const Geo &g) { return sizeof(cplx<T>) * (kMaxN + 2 * kZCols * (g.n3 + 1)); }
template <typename T> size_t plane_smem(const Geo &g) {
  return sizeof(cplx<T>) * (2 * kMaxN + (size_t)g.n2 * g.pitch) + sizeof(int) * g.nxact;
}

template <typename T>
void set_fft_smem_limits(const Geo &g) {
  const int zs = (int)zpass_smem<T>(g), ps = (int)plane_smem<T>(g);
  raise_smem_limit(k_zpass_g2r<T, false, 0>, (size_t)(zs));
  raise_smem_limit(k_zpass_g2r<T, true, 0>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_STORE, 0>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_HSHIFT, 0>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_DRHO, 0>, (size_t)(zs));
  raise_smem_limit(k_plane<T, OP_VLOC>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_G2R>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_PROD_R2G>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_ACCUM>, (size_t)(ps));
  set_plane_fast_limits<T>(g);
  set_zpass_fast_limits<T>(g);
  if constexpr (!std::is_same<T, double>::value) set_zpass_more_limits<T>(g);
}

// the further compile-time n3 sizes exist for float and double-float
template <typename T> static constexpr bool has_more() { return !std::is_same<T, double>::value; }

template <typename T>
void launch_zpass_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (nvec <= 0) return;
  if (zpass_fast_g2r<T>(f, X, nvec, cb, st)) return;
  if constexpr (has_more<T>())
    if (zpass_more_g2r<T>(f, X, nvec, cb, st)) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, false, 0>, dim3(grid), dim3(kThreads), zpass_smem<T>(f.g), st, X, nvec, f.g, f.P3,
         f.tw3, cb, PDir<T>());
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void launch_zpass_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (nvec <= 0) return;
  if (zpass_fast_g2r_dir<T>(f, d, nvec, cb, st)) return;
  if constexpr (has_more<T>())
    if (zpass_more_g2r_dir<T>(f, d, nvec, cb, st)) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, true, 0>, dim3(grid), dim3(kThreads), zpass_smem<T>(f.g), st,
         (const cplx<T> *)d.p, nvec, f.g, f.P3, f.tw3, cb, d);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void launch_zpass_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
  if (nvec <= 0) return;
  if (zpass_fast_r2g<T>(f, epi, cb, nvec, ea, st)) return;
  if constexpr (has_more<T>())
    if (zpass_more_r2g<T>(f, epi, cb, nvec, ea, st)) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  const size_t sm = zpass_smem<T>(f.g);
  if (epi == EPI_STORE) launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_STORE, 0>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
  else if (epi == EPI_HSHIFT) launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_HSHIFT, 0>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
  else launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_DRHO, 0>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void launch_plane(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st) {
  if (nblk <= 0) return;
  if (launch_plane_fast<T>(f, op, nblk, pa, st)) return;
  dim3 grid(nblk, f.g.n3);
  const size_t sm = plane_smem<T>(f.g);
  switch (op) {
    case OP_VLOC: launch("plane_vloc", bits_of<T>(), k_plane<T, OP_VLOC>, dim3(grid), dim3(kThreads), sm, st, f.g, f.P1, f.P2, f.tw1, f.tw2, pa); break;
    case OP_G2R: launch("plane_g2r", bits_of<T>(), k_plane<T, OP_G2R>, dim3(grid), dim3(kThreads), sm, st, f.g, f.P1, f.P2, f.tw1, f.tw2, pa); break;
    case OP_PROD_R2G: launch("plane_prod", bits_of<T>(), k_plane<T, OP_PROD_R2G>, dim3(grid), dim3(kThreads), sm, st, f.g, f.P1, f.P2, f.tw1, f.tw2, pa); break;
    default: launch("plane_accum", bits_of<T>(), k_plane<T, OP_ACCUM>, dim3(grid), dim3(kThreads), sm, st, f.g, f.P1, f.P2, f.tw1, f.tw2, pa); break;
  }
  WDF_CUDA_TRY(cudaGetLastError());
}

#define WDF_INST(T)                                                                                         \
  template void set_fft_smem_limits<T>(const Geo &);                                                        \
  template size_t plane_smem<T>(const Geo &);                                                               \
  template size_t zpass_smem<T>(const Geo &);                                                               \
  template void launch_zpass_g2r<T>(const FftCtx<T> &, const cplx<T> *, int, cplx<T> *, cudaStream_t);      \
  template void launch_zpass_g2r_dir<T>(const FftCtx<T> &, const PDir<T> &, int, cplx<T> *, cudaStream_t);  \
  template void launch_zpass_r2g<T>(const FftCtx<T> &, int, const cplx<T> *, int, const EpiArgs<T> &,       \
                                    cudaStream_t);                                                          \
  template void launch_plane<T>(const FftCtx<T> &, int, int, const PlaneArgs<T> &, cudaStream_t);
WDF_INST(double)
WDF_INST(float)
WDF_INST(df64)
#undef WDF_INST

}  // namespace wdf

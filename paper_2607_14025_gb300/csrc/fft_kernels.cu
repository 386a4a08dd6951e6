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

namespace wdf {

constexpr int kThreads = 256;

static __device__ __forceinline__ int wrap(int z, int n) {
  int m = z % n;
  return m < 0 ? m + n : m;
}

// ---------------------------------------------------------------------------------------------
// n3 transforms, G -> r

template <typename T, bool DIR>
__global__ void __launch_bounds__(kThreads) k_zpass_g2r(const cplx<T> *X, int nvec, Geo g, Plan1D P3,
                                                         const cplx<T> *__restrict__ tw3, cplx<T> *__restrict__ cb, PDir<T> pd) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T> *tw = reinterpret_cast<cplx<T> *>(smraw);
  cplx<T> *sm = tw + kMaxN;
  const int q = blockIdx.x;
  const int k0 = blockIdx.y * kZCols;
  const int n3 = g.n3, pitch = n3 + 1, nlines = 2 * kZCols;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = tw3[i];
  for (int i = threadIdx.x; i < nlines * pitch; i += blockDim.x) sm[i] = mkc<T>(0, 0);
  __syncthreads();
  const int kend = min(k0 + kZCols, g.K);
  const int e0 = g.col_off[k0], e1 = g.col_off[kend];
  const cplx<T> *xa = X + (size_t)(2 * q) * g.ld;
  const cplx<T> *xb = (2 * q + 1 < nvec) ? X + (size_t)(2 * q + 1) * g.ld : nullptr;
  const int sa = 2 * q, sb = 2 * q + 1;
  const bool upa = DIR && pd.active[sa], upb = DIR && xb && pd.active[sb];
  const T *Ka = (DIR && pd.K) ? pd.K + (size_t)pd.vidx[sa] * g.ld : nullptr;
  const T *Kb = (DIR && pd.K && xb) ? pd.K + (size_t)pd.vidx[sb] * g.ld : nullptr;
  const T ba = DIR ? (T)pd.beta[sa] : (T)0, bbeta = (DIR && xb) ? (T)pd.beta[sb] : (T)0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int k = g.e_col[e], c = k - k0, z = g.e_z[e];
    cplx<T> a = xa[e];
    cplx<T> b = xb ? xb[e] : mkc<T>(0, 0);
    if (DIR) {  // p = K r + beta p, written back (each element belongs to exactly one block)
      if (upa) {
        const cplx<T> rv = pd.r[(size_t)sa * g.ld + e];
        const T kk = Ka ? Ka[e] : (T)1;
        a = mkc<T>(kk * rv.x + ba * a.x, kk * rv.y + ba * a.y);
        pd.p[(size_t)sa * g.ld + e] = a;
      }
      if (upb) {
        const cplx<T> rv = pd.r[(size_t)sb * g.ld + e];
        const T kk = Kb ? Kb[e] : (T)1;
        b = mkc<T>(kk * rv.x + bbeta * b.x, kk * rv.y + bbeta * b.y);
        pd.p[(size_t)sb * g.ld + e] = b;
      }
    }
    sm[c * pitch + g.pos3[wrap(z, n3)]] = mkc<T>(a.x - b.y, a.y + b.x);  // a + i b at G
    if (k != 0) sm[(kZCols + c) * pitch + g.pos3[wrap(-z, n3)]] = mkc<T>(a.x + b.y, b.x - a.y);  // at -G
  }
  __syncthreads();
  fft_lines<T, true>(sm, nlines, nullptr, pitch, 1, P3, tw);
  cplx<T> *out = cb + (size_t)q * n3 * g.ldcb;
  const int ncol = kend - k0;
  for (int it = threadIdx.x; it < n3 * nlines; it += blockDim.x) {
    const int z = it / nlines, c2 = it - z * nlines;
    if (c2 < kZCols) {
      if (c2 < ncol) out[(size_t)z * g.ldcb + k0 + c2] = sm[c2 * pitch + z];
    } else {
      const int c = c2 - kZCols, k = k0 + c;
      if (c < ncol && k >= 1) out[(size_t)z * g.ldcb + g.K - 1 + k] = sm[c2 * pitch + z];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// n3 transforms, r -> G, with the Gamma unpacking and an epilogue

template <typename T, int EPI>
__global__ void __launch_bounds__(kThreads) k_zpass_r2g(const cplx<T> *__restrict__ cb, int nvec, Geo g, Plan1D P3,
                                                         const cplx<T> *__restrict__ tw3, EpiArgs<T> ea) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T> *tw = reinterpret_cast<cplx<T> *>(smraw);
  cplx<T> *sm = tw + kMaxN;
  const int q = blockIdx.x;
  const int k0 = blockIdx.y * kZCols;
  const int n3 = g.n3, pitch = n3 + 1, nlines = 2 * kZCols;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = tw3[i];
  const int kend = min(k0 + kZCols, g.K);
  const int ncol = kend - k0;
  const cplx<T> *in = cb + (size_t)q * n3 * g.ldcb;
  for (int it = threadIdx.x; it < n3 * nlines; it += blockDim.x) {
    const int z = it / nlines, c2 = it - z * nlines;
    cplx<T> v = mkc<T>(0, 0);
    if (c2 < kZCols) {
      if (c2 < ncol) v = in[(size_t)z * g.ldcb + k0 + c2];
    } else {
      const int c = c2 - kZCols, k = k0 + c;
      if (c < ncol && k >= 1) v = in[(size_t)z * g.ldcb + g.K - 1 + k];
    }
    sm[c2 * pitch + z] = v;
  }
  __syncthreads();
  fft_lines<T, false>(sm, nlines, nullptr, pitch, 1, P3, tw);
  const int e0 = g.col_off[k0], e1 = g.col_off[kend];
  const int sa = 2 * q, sb = 2 * q + 1;
  const bool hasb = sb < nvec;
  const T sc = ea.scale;
  T sha = 0, shb = 0;  // per-vector shifts, converted once (the stores below may alias the array)
  if (EPI == EPI_HSHIFT) {
    sha = (T)ea.shift[sa];
    if (hasb) shb = (T)ea.shift[sb];
  }
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int k = g.e_col[e], c = k - k0, z = g.e_z[e];
    const cplx<T> g1 = sm[c * pitch + g.pos3[wrap(z, n3)]];
    const cplx<T> g2 = sm[(k == 0 ? c : kZCols + c) * pitch + g.pos3[wrap(-z, n3)]];
    // a(G) = (F(G) + conj F(-G)) / 2,  b(G) = (F(G) - conj F(-G)) / (2i)
    const cplx<T> a = mkc<T>((T)0.5 * sc * (g1.x + g2.x), (T)0.5 * sc * (g1.y - g2.y));
    const cplx<T> b = mkc<T>((T)0.5 * sc * (g1.y + g2.y), (T)0.5 * sc * (g2.x - g1.x));
    if (EPI == EPI_STORE) {
      ea.Y[(size_t)sa * g.ld + e] = a;
      if (hasb) ea.Y[(size_t)sb * g.ld + e] = b;
    } else if (EPI == EPI_HSHIFT) {
      // Y = V x (unpacked) + (1/2 |G|^2 - shift_s) x
      const T kin = (T)(0.5 * g.g2[e]);
      {
        const cplx<T> xv = ea.X[(size_t)sa * g.ld + e];
        const T d = kin - sha;
        ea.Y[(size_t)sa * g.ld + e] = mkc<T>(a.x + d * xv.x, a.y + d * xv.y);
      }
      if (hasb) {
        const cplx<T> xv = ea.X[(size_t)sb * g.ld + e];
        const T d = kin - shb;
        ea.Y[(size_t)sb * g.ld + e] = mkc<T>(b.x + d * xv.x, b.y + d * xv.y);
      }
    } else {  // EPI_DRHO: Y = drho, Y2 = v^1/2 drho
      const T vh = (T)ea.vhalf[e];
      ea.Y[(size_t)sa * g.ld + e] = a;
      ea.Y2[(size_t)sa * g.ld + e] = cscal<T>(a, vh);
      if (hasb) {
        ea.Y[(size_t)sb * g.ld + e] = b;
        ea.Y2[(size_t)sb * g.ld + e] = cscal<T>(b, vh);
      }
    }
  }
}

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
  raise_smem_limit(k_zpass_g2r<T, false>, (size_t)(zs));
  raise_smem_limit(k_zpass_g2r<T, true>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_STORE>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_HSHIFT>, (size_t)(zs));
  raise_smem_limit(k_zpass_r2g<T, EPI_DRHO>, (size_t)(zs));
  raise_smem_limit(k_plane<T, OP_VLOC>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_G2R>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_PROD_R2G>, (size_t)(ps));
  raise_smem_limit(k_plane<T, OP_ACCUM>, (size_t)(ps));
  set_plane_fast_limits<T>(g);
}

template <typename T>
void launch_zpass_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (nvec <= 0) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, false>, dim3(grid), dim3(kThreads), zpass_smem<T>(f.g), st, X, nvec, f.g, f.P3,
         f.tw3, cb, PDir<T>());
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void launch_zpass_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (nvec <= 0) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, true>, dim3(grid), dim3(kThreads), zpass_smem<T>(f.g), st,
         (const cplx<T> *)d.p, nvec, f.g, f.P3, f.tw3, cb, d);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void launch_zpass_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
  if (nvec <= 0) return;
  dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  const size_t sm = zpass_smem<T>(f.g);
  if (epi == EPI_STORE) launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_STORE>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
  else if (epi == EPI_HSHIFT) launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_HSHIFT>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
  else launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_DRHO>, dim3(grid), dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
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

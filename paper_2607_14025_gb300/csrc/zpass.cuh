// n3 transforms of the batched Gamma-point 3-D FFT (see fft_kernels.cu for the data model):
// k_zpass_g2r packs two real vectors per complex column and transforms the disk columns along n3
// into the column buffer; k_zpass_r2g transforms back, unpacks and applies an epilogue. N3 = 0
// is the generic mixed-radix kernel (runtime plan, in place on digit-reversed input); N3 > 0 a
// compile-time Stockham transform in natural order (stockham.cuh).
#pragma once

#include "fft.cuh"
#include "kernels.cuh"
#include "stockham.cuh"

namespace wdf {

constexpr int kThreads = 256;

static __device__ __forceinline__ int wrap(int z, int n) {
  int m = z % n;
  return m < 0 ? m + n : m;
}

// ---------------------------------------------------------------------------------------------
// n3 transforms, G -> r

template <typename T, bool DIR, int N3>
__global__ void __launch_bounds__(kThreads) k_zpass_g2r(const cplx<T> *X, int nvec, Geo g, Plan1D P3,
                                                         const cplx<T> *__restrict__ tw3, cplx<T> *__restrict__ cb, PDir<T> pd) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T> *tw = reinterpret_cast<cplx<T> *>(smraw);
  cplx<T> *sm = tw + kMaxN;
  const int q = blockIdx.x;
  const int k0 = blockIdx.y * kZCols;
  const int n3 = N3 > 0 ? N3 : g.n3, pitch = n3 + 1, nlines = 2 * kZCols;
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
    // the generic transform works in place on digit-reversed input; the compile-time one takes
    // natural order
    const int zp = N3 > 0 ? wrap(z, n3) : g.pos3[wrap(z, n3)], zm = N3 > 0 ? wrap(-z, n3) : g.pos3[wrap(-z, n3)];
    sm[c * pitch + zp] = mkc<T>(a.x - b.y, a.y + b.x);                  // a + i b at G
    if (k != 0) sm[(kZCols + c) * pitch + zm] = mkc<T>(a.x + b.y, b.x - a.y);  // at -G
  }
  __syncthreads();
  if constexpr (N3 > 0) zlines_fft<T, N3, 1, 2 * kZCols, N3 + 1, kThreads>(sm, tw);
  else fft_lines<T, true>(sm, nlines, nullptr, pitch, 1, P3, tw);
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

template <typename T, int EPI, int N3>
__global__ void __launch_bounds__(kThreads) k_zpass_r2g(const cplx<T> *__restrict__ cb, int nvec, Geo g, Plan1D P3,
                                                         const cplx<T> *__restrict__ tw3, EpiArgs<T> ea) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T> *tw = reinterpret_cast<cplx<T> *>(smraw);
  cplx<T> *sm = tw + kMaxN;
  const int q = blockIdx.x;
  const int k0 = blockIdx.y * kZCols;
  const int n3 = N3 > 0 ? N3 : g.n3, pitch = n3 + 1, nlines = 2 * kZCols;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw[i] = tw3[i];
  const int kend = min(k0 + kZCols, g.K);
  const int ncol = kend - k0;
  const cplx<T> *in = cb + (size_t)q * n3 * g.ldcb;
  // column-buffer element `it` of this block: (z, c2) with c2 < kZCols the rep columns, the rest
  // their mirrors; zero outside the sphere's columns
  auto fetch = [&](int it) {
    const int z = it / nlines, c2 = it - z * nlines;
    cplx<T> v = mkc<T>(0, 0);
    if (c2 < kZCols) {
      if (c2 < ncol) v = in[(size_t)z * g.ldcb + k0 + c2];
    } else {
      const int c = c2 - kZCols, k = k0 + c;
      if (c < ncol && k >= 1) v = in[(size_t)z * g.ldcb + g.K - 1 + k];
    }
    return v;
  };
  if constexpr (N3 > 0) {
    // all of a thread's loads first (a compile-time count), then the shared-memory stores: the
    // loads are in flight together instead of one at a time
    constexpr int TOT = N3 * 2 * kZCols, NIT = (TOT + kThreads - 1) / kThreads;
    cplx<T> vv[NIT];
#pragma unroll
    for (int u = 0; u < NIT; ++u) {
      const int it = threadIdx.x + u * kThreads;
      vv[u] = (TOT % kThreads == 0 || it < TOT) ? fetch(it) : mkc<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < NIT; ++u) {
      const int it = threadIdx.x + u * kThreads;
      if (TOT % kThreads == 0 || it < TOT) {
        const int z = it / nlines, c2 = it - z * nlines;
        sm[c2 * pitch + z] = vv[u];
      }
    }
  } else {
    for (int it = threadIdx.x; it < n3 * nlines; it += blockDim.x) {
      const int z = it / nlines, c2 = it - z * nlines;
      sm[c2 * pitch + z] = fetch(it);
    }
  }
  __syncthreads();
  if constexpr (N3 > 0) zlines_fft<T, N3, -1, 2 * kZCols, N3 + 1, kThreads>(sm, tw);
  else fft_lines<T, false>(sm, nlines, nullptr, pitch, 1, P3, tw);
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
    const int zp = N3 > 0 ? wrap(z, n3) : g.pos3[wrap(z, n3)], zm = N3 > 0 ? wrap(-z, n3) : g.pos3[wrap(-z, n3)];
    const cplx<T> g1 = sm[c * pitch + zp];
    const cplx<T> g2 = sm[(k == 0 ? c : kZCols + c) * pitch + zm];
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

}  // namespace wdf

// Plane kernels specialised for compile-time grid sizes (n1 = n2 = N).
//
// Same operations as k_plane in fft_kernels.cu (one z plane of one pair per block: n2 transforms
// of the occupied n1 columns, n1 transforms of every row, the pointwise work and the way back),
// organised for throughput:
//  * Stockham passes with the radix in registers (radix 8 first, then 4, 5, 3, 2): natural order
//    in and out, so the column buffer is gathered and scattered directly (table jidx[y][x]) with
//    no zeroing or digit-reversal passes. Pass (radix R, stride Ls): thread j reads
//    in[j + r N/R], multiplies by w^(r k / (Ls R)) with k = j mod Ls, does an R-point DFT and
//    writes out[(j / Ls) Ls R + k + r Ls]; in place, with a barrier between reads and writes.
//  * After the last inverse pass along n1 a thread holds the elements j + r N/R of its rows,
//    exactly the inputs of the first forward pass when that pass uses the same radix: the
//    pointwise product (V_loc, or psi_v times dV) and the orbital sum of the density response
//    stay in registers.
//  * All index arithmetic is on compile-time sizes.
#include <cstdlib>

#include "fft.cuh"
#include "kernels.cuh"
#include "stockham.cuh"
#include "plane_reg.cuh"

namespace wdf {

template <int N> struct PlaneShape {
  static constexpr int threads = (N * N / 16 < 64) ? 64 : ((N * N / 16 + 31) / 32 * 32 > 1024 ? 1024 : (N * N / 16 + 31) / 32 * 32);
  static constexpr int pitch = N + 1;
};

// Pieces of one pass over nlines lines of length N (line l starts at base(l) = lbase[l] or
// l * lpitch, element t at base + t * es): pass_load reads the R inputs of each task, pass_compute
// twiddles and transforms them in registers, pass_store writes the outputs. TPT tasks per thread;
// task t -> line t % nlines, butterfly j = t / nlines.
template <typename T, int N, int R, int LS, int SIGN, int TPT>
__device__ __forceinline__ void pass_compute(cplx<T> (&v)[TPT][R], int nlines, const cplx<T> *tw) {
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    if (t < nlines * (N / R)) {
      const int j = t / nlines;
      const int k = j % LS;
      if constexpr (LS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const cplx<T> w = tw[(r * k * (N / (LS * R))) % N];
          v[u][r] = (SIGN > 0) ? cmul<T>(v[u][r], w) : cmulc<T>(v[u][r], w);
        }
      }
      dft_reg<T, R, SIGN>(v[u]);
    }
  }
}

template <typename T, int N, int R, int TPT>
__device__ __forceinline__ void pass_load(cplx<T> (&v)[TPT][R], const cplx<T> *tile, int nlines, const int *lbase, int lpitch,
                                          int es) {
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    if (t < nlines * (N / R)) {
      const int l = t % nlines, j = t / nlines;
      const int b = lbase ? lbase[l] : l * lpitch;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u][r] = tile[b + (j + r * (N / R)) * es];
    }
  }
}

template <typename T, int N, int R, int LS, int TPT>
__device__ __forceinline__ void pass_store(const cplx<T> (&v)[TPT][R], cplx<T> *tile, int nlines, const int *lbase, int lpitch,
                                           int es) {
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    if (t < nlines * (N / R)) {
      const int l = t % nlines, j = t / nlines;
      const int b = lbase ? lbase[l] : l * lpitch;
      const int k = j % LS;
      const int o = (j / LS) * LS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) tile[b + (o + r * LS) * es] = v[u][r];
    }
  }
}

// full in-place pass through the tile: load, barrier-free compute, barrier, store, barrier
template <typename T, int N, int P, int SIGN, int THREADS>
__device__ __forceinline__ void tile_pass(cplx<T> *tile, int nlines, const int *lbase, int lpitch, int es, const cplx<T> *tw) {
  constexpr int R = SIGN > 0 ? rad_at(N, P) : frad_at(N, P);
  constexpr int LS = SIGN > 0 ? ls_at(N, P) : fls_at(N, P);
  constexpr int TPT = cdiv(N * (N / R), THREADS);
  cplx<T> v[TPT][R];
  pass_load<T, N, R, TPT>(v, tile, nlines, lbase, lpitch, es);
  pass_compute<T, N, R, LS, SIGN, TPT>(v, nlines, tw);
  __syncthreads();
  pass_store<T, N, R, LS, TPT>(v, tile, nlines, lbase, lpitch, es);
  __syncthreads();
}

// inverse transform along n2 of the active n1 columns; the first pass gathers from the column
// buffer slice cbz through jidx (disk column of each (y, x), or -1)
template <typename T, int N, int THREADS>
__device__ __forceinline__ void y_inverse(cplx<T> *tile, const cplx<T> *__restrict__ cbz, const int *__restrict__ jidx, const int *xact,
                                          int nx, const cplx<T> *tw) {
  constexpr int P = N + 1;
  {
    constexpr int R = rad_at(N, 0);
    constexpr int TPT = cdiv(N * (N / R), THREADS);
    cplx<T> v[TPT][R];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < nx * (N / R)) {
        const int l = t % nx, j = t / nx;
        const int x = xact[l];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int y = j + r * (N / R);
          const int jj = __ldg(jidx + y * N + x);
          v[u][r] = jj >= 0 ? cbz[jj] : mkc<T>(0, 0);
        }
      }
    }
    pass_compute<T, N, R, 1, 1, TPT>(v, nx, tw);
    pass_store<T, N, R, 1, TPT>(v, tile, nx, xact, 0, P);  // nobody reads the tile yet
    __syncthreads();
  }
  if constexpr (nrad(N) > 1) tile_pass<T, N, 1, 1, THREADS>(tile, nx, xact, 0, P, tw);
  if constexpr (nrad(N) > 2) tile_pass<T, N, 2, 1, THREADS>(tile, nx, xact, 0, P, tw);
  if constexpr (nrad(N) > 3) tile_pass<T, N, 3, 1, THREADS>(tile, nx, xact, 0, P, tw);
}

// forward transform along n2 of the active columns; the last pass scatters to cbz through jidx
template <typename T, int N, int THREADS>
__device__ __forceinline__ void y_forward(cplx<T> *tile, cplx<T> *__restrict__ cbz, const int *__restrict__ jidx, const int *xact, int nx,
                                          const cplx<T> *tw) {
  constexpr int P = N + 1;
  constexpr int NR = nrad(N);
  if constexpr (NR > 1) tile_pass<T, N, 0, -1, THREADS>(tile, nx, xact, 0, P, tw);
  if constexpr (NR > 2) tile_pass<T, N, 1, -1, THREADS>(tile, nx, xact, 0, P, tw);
  if constexpr (NR > 3) tile_pass<T, N, 2, -1, THREADS>(tile, nx, xact, 0, P, tw);
  {
    constexpr int PL = NR - 1;
    constexpr int R = frad_at(N, PL);
    constexpr int LS = fls_at(N, PL);
    constexpr int TPT = cdiv(N * (N / R), THREADS);
    cplx<T> v[TPT][R];
    pass_load<T, N, R, TPT>(v, tile, nx, xact, 0, P);
    pass_compute<T, N, R, LS, -1, TPT>(v, nx, tw);
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < nx * (N / R)) {
        const int l = t % nx, j = t / nx;
        const int x = xact[l];
        const int k = j % LS;
        const int o = (j / LS) * LS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int y = o + r * LS;
          const int jj = __ldg(jidx + y * N + x);
          if (jj >= 0) cbz[jj] = v[u][r];
        }
      }
    }
  }
}

// inverse along n1 of every row, all passes but the last through the tile; the last pass leaves
// its results in registers: thread task t -> row t % N, elements j + r N / RL (j = t / N).
// Inactive columns (outside the sphere's n1 range) read as zero in the first pass.
template <typename T, int N, int THREADS, int RL, int TPL>
__device__ __forceinline__ void x_inverse_to_regs(cplx<T> (&v)[TPL][RL], cplx<T> *tile, int xmax, const cplx<T> *tw) {
  constexpr int P = N + 1;
  constexpr int NR = nrad(N);
  static_assert(RL == rad_at(N, NR - 1), "last radix");
  if constexpr (NR > 1) {
    constexpr int R = rad_at(N, 0);
    constexpr int TPT = cdiv(N * (N / R), THREADS);
    cplx<T> w[TPT][R];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < N * (N / R)) {
        const int l = t % N, j = t / N;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int x = j + r * (N / R);
          w[u][r] = (x <= xmax || x >= N - xmax) ? tile[l * P + x] : mkc<T>(0, 0);
        }
      }
    }
    pass_compute<T, N, R, 1, 1, TPT>(w, N, tw);
    __syncthreads();
    pass_store<T, N, R, 1, TPT>(w, tile, N, nullptr, P, 1);
    __syncthreads();
    if constexpr (NR > 2) tile_pass<T, N, 1, 1, THREADS>(tile, N, nullptr, P, 1, tw);
    if constexpr (NR > 3) tile_pass<T, N, 2, 1, THREADS>(tile, N, nullptr, P, 1, tw);
    pass_load<T, N, RL, TPL>(v, tile, N, nullptr, P, 1);
    pass_compute<T, N, RL, ls_at(N, NR - 1), 1, TPL>(v, N, tw);
  } else {
#pragma unroll
    for (int u = 0; u < TPL; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < N * (N / RL)) {
        const int l = t % N, j = t / N;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int x = j + r * (N / RL);
          v[u][r] = (x <= xmax || x >= N - xmax) ? tile[l * P + x] : mkc<T>(0, 0);
        }
      }
    }
    pass_compute<T, N, RL, 1, 1, TPL>(v, N, tw);
  }
}

// forward along n1 of every row starting from registers (the first forward pass uses the same
// radix as the last inverse one), the rest through the tile
template <typename T, int N, int THREADS, int RL, int TPL>
__device__ __forceinline__ void x_forward_from_regs(cplx<T> (&v)[TPL][RL], cplx<T> *tile, const cplx<T> *tw) {
  constexpr int P = N + 1;
  constexpr int NR = nrad(N);
  static_assert(RL == frad_at(N, 0), "first forward radix");
  pass_compute<T, N, RL, 1, -1, TPL>(v, N, tw);
  __syncthreads();  // every thread has loaded its inputs (from the tile or from registers)
  pass_store<T, N, RL, 1, TPL>(v, tile, N, nullptr, P, 1);
  __syncthreads();
  if constexpr (NR > 1) tile_pass<T, N, 1, -1, THREADS>(tile, N, nullptr, P, 1, tw);
  if constexpr (NR > 2) tile_pass<T, N, 2, -1, THREADS>(tile, N, nullptr, P, 1, tw);
  if constexpr (NR > 3) tile_pass<T, N, 3, -1, THREADS>(tile, N, nullptr, P, 1, tw);
}

template <typename T, int N, int OP>
__global__ void __launch_bounds__(PlaneShape<N>::threads) k_plane_fast(Geo g, const cplx<T> *__restrict__ twg,
                                                                        const int *__restrict__ jidx, PlaneArgs<T> pa) {
  constexpr int THREADS = PlaneShape<N>::threads;
  constexpr int P = N + 1;
  constexpr int NR = nrad(N);
  constexpr int RL = rad_at(N, NR - 1);
  constexpr int TPL = cdiv(N * (N / RL), THREADS);
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T> *tw = reinterpret_cast<cplx<T> *>(smraw);
  cplx<T> *tile = tw + N;
  int *xact = reinterpret_cast<int *>(tile + N * P);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < g.nxact; i += blockDim.x) xact[i] = g.xactn[i];
  __syncthreads();
  const int nx = g.nxact;
  const int xmax = g.xmax;
  const int z = blockIdx.y;
  constexpr size_t plane = (size_t)N * N;
  const size_t cbpair = (size_t)g.n3 * g.ldcb;
  cplx<T> v[TPL][RL];

  if (OP == OP_VLOC || OP == OP_G2R) {
    const int q = blockIdx.x;
    cplx<T> *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    y_inverse<T, N, THREADS>(tile, cbz, jidx, xact, nx, tw);
    x_inverse_to_regs<T, N, THREADS, RL, TPL>(v, tile, xmax, tw);
    if (OP == OP_G2R) {
      cplx<T> *out = pa.grid + (size_t)q * g.n3 * plane + (size_t)z * plane;
#pragma unroll
      for (int u = 0; u < TPL; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < N * (N / RL)) {
          const int l = t % N, j = t / N;
#pragma unroll
          for (int r = 0; r < RL; ++r) out[l * N + j + r * (N / RL)] = v[u][r];
        }
      }
      return;
    }
    const T *vz = pa.field + (size_t)z * plane;
#pragma unroll
    for (int u = 0; u < TPL; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < N * (N / RL)) {
        const int l = t % N, j = t / N;
#pragma unroll
        for (int r = 0; r < RL; ++r) v[u][r] = cscal<T>(v[u][r], vz[l * N + j + r * (N / RL)]);
      }
    }
    x_forward_from_regs<T, N, THREADS, RL, TPL>(v, tile, tw);
    y_forward<T, N, THREADS>(tile, cbz, jidx, xact, nx, tw);
  } else if (OP == OP_PROD_R2G) {
    // pair q = pp * nocc + v:  F(r) = psi_v(r) (dV_2pp + i dV_2pp+1)(r)
    const int q = blockIdx.x;
    const int vo = q % pa.nocc, pp = q / pa.nocc;
    const T *psi = pa.field + (size_t)vo * g.n3 * plane + (size_t)z * plane;
    const cplx<T> *dv = pa.grid + (size_t)pp * g.n3 * plane + (size_t)z * plane;
#pragma unroll
    for (int u = 0; u < TPL; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < N * (N / RL)) {
        const int l = t % N, j = t / N;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int i = l * N + j + r * (N / RL);
          v[u][r] = cscal<T>(dv[i], psi[i]);
        }
      }
    }
    cplx<T> *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    x_forward_from_regs<T, N, THREADS, RL, TPL>(v, tile, tw);
    y_forward<T, N, THREADS>(tile, cbz, jidx, xact, nx, tw);
  } else {  // OP_ACCUM: acc(r) = sum_v psi_v(r) G2R(cb[pp * nocc + v]), held in registers
    const int pp = blockIdx.x;
    cplx<T> acc[TPL][RL];
#pragma unroll
    for (int u = 0; u < TPL; ++u)
#pragma unroll
      for (int r = 0; r < RL; ++r) acc[u][r] = mkc<T>(0, 0);
    for (int vo = 0; vo < pa.nocc; ++vo) {
      const cplx<T> *cbz = pa.cb + ((size_t)pp * pa.nocc + vo) * cbpair + (size_t)z * g.ldcb;
      y_inverse<T, N, THREADS>(tile, cbz, jidx, xact, nx, tw);
      x_inverse_to_regs<T, N, THREADS, RL, TPL>(v, tile, xmax, tw);
      const T *psi = pa.field + (size_t)vo * g.n3 * plane + (size_t)z * plane;
#pragma unroll
      for (int u = 0; u < TPL; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < N * (N / RL)) {
          const int l = t % N, j = t / N;
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const T s = psi[l * N + j + r * (N / RL)];
            acc[u][r].x += s * v[u][r].x;
            acc[u][r].y += s * v[u][r].y;
          }
        }
      }
      __syncthreads();  // the next orbital reuses the tile
    }
    cplx<T> *cbz = pa.cb2 + (size_t)pp * cbpair + (size_t)z * g.ldcb;
    x_forward_from_regs<T, N, THREADS, RL, TPL>(acc, tile, tw);
    y_forward<T, N, THREADS>(tile, cbz, jidx, xact, nx, tw);
  }
}

// ---------------------------------------------------------------------------------------------
// FP32 V_loc plane kernel with whole lines in registers (n1 = n2 = N = 8 R2, R2 in {3, 4, 5, 8}).
// One thread owns one line of N complex values: a four-step DFT with static register indices
// (8-point DFTs over stride-R2 subsequences, twiddles, R2-point DFTs over consecutive slots).
// The inverse takes natural order and leaves X[k1 + 8 k2] in slot k2 + R2 k1; the forward
// transform takes exactly that permuted order and returns natural order, so the n1 inverse, the
// V_loc product and the n1 forward transform of a row never leave registers. Shared memory only
// carries the two transpositions between columns (n2 transforms) and rows (n1 transforms).

template <int N>
__global__ void __launch_bounds__(N) k_plane_reg(Geo g, const float2 *__restrict__ twg, const int *__restrict__ jidx,
                                                 PlaneArgs<float> pa) {
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 *tw = reinterpret_cast<float2 *>(smraw);
  float2 *tile = tw + N;
  float *vsm = reinterpret_cast<float *>(tile + N * P);
  int *xact = reinterpret_cast<int *>(vsm + N * P);
  const int t = threadIdx.x, z = blockIdx.y, q = blockIdx.x;
  const int nx = g.nxact, xmax = g.xmax;
  tw[t] = twg[t];
  for (int i = t; i < nx; i += N) xact[i] = g.xactn[i];
  const float4 *vz = reinterpret_cast<const float4 *>(pa.field + (size_t)z * N * N);
  for (int i = t; i < N * N / 4; i += N) {  // 16-byte loads, padded rows
    const int row = i / (N / 4), c = 4 * (i % (N / 4));
    const float4 w = vz[i];
    vsm[row * P + c] = w.x;
    vsm[row * P + c + 1] = w.y;
    vsm[row * P + c + 2] = w.z;
    vsm[row * P + c + 3] = w.w;
  }
  __syncthreads();
  float2 *cbz = pa.cb + (size_t)q * g.n3 * g.ldcb + (size_t)z * g.ldcb;
  float2 v[N];
  if (t < nx) {  // inverse along n2 of occupied column x
    const int x = xact[t];
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int jj = __ldg(jidx + y * N + x);
      v[y] = jj >= 0 ? cbz[jj] : mkc<float>(0.f, 0.f);
    }
    line_inverse<N>(v, tw);
#pragma unroll
    for (int s = 0; s < N; ++s) tile[perm_index<N>(s) * P + x] = v[s];
  }
  __syncthreads();
  {  // row y = t: inverse along n1, V_loc, forward along n1 (each thread touches its own row only)
    const int y = t;
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = (x <= xmax || x >= N - xmax) ? tile[y * P + x] : mkc<float>(0.f, 0.f);
    line_inverse<N>(v, tw);
#pragma unroll
    for (int s = 0; s < N; ++s) v[s] = cscal<float>(v[s], vsm[y * P + perm_index<N>(s)]);
    line_forward<N>(v, tw);
#pragma unroll
    for (int x = 0; x < N; ++x)
      if (x <= xmax || x >= N - xmax) tile[y * P + x] = v[x];
  }
  __syncthreads();
  if (t < nx) {  // forward along n2 of occupied column x, scattered back to the column buffer
    const int x = xact[t];
#pragma unroll
    for (int s = 0; s < N; ++s) v[s] = tile[perm_index<N>(s) * P + x];
    line_forward<N>(v, tw);
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int jj = __ldg(jidx + y * N + x);
      if (jj >= 0) cbz[jj] = v[y];
    }
  }
}

// Two threads per line, N = 64 = 8 x 8: lanes 2i and 2i+1 share a line, each holding 32 values
// in v[g][e] (g < 4, e < 8). Inverse: lane h first holds x[4h + g + 8 n1] at v[g][n1], transforms
// the 4 radix-8 groups n2 = 4h + g over n1 with twiddles w^(n2 k1), exchanges the 16 values whose
// k1 belongs to the other lane (one shuffle each way per value), and transforms over n2; the
// result X[4h + j + 8 k2] sits at v[k2 % 4][4 (k2 / 4) + j]. The forward transform starts from
// that distribution (no exchange before its first stage) and ends with Y[4h + g + 8 q1] at
// v[g][q1], the inverse's input distribution. Half the registers of the one-thread line, so
// twice the warps per SM at the same shared memory.
__device__ __forceinline__ void pair_exchange(float2 (&v)[4][8], int h, bool fwd) {
  // inverse: lane h sends (n2 = 4h + g, k1 = 4(1-h) + j) from v[g][4(1-h) + j] and receives the
  // partner's (n2 = 4(1-h) + g, k1 = 4h + j) into that slot; forward: the same slots with the
  // roles of k1 and q2 (see the caller), so both directions exchange v[g][4(1-h) + j]
  (void)fwd;
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float2 &a = v[g][j], &b = v[g][4 + j];
      const float2 send = h ? a : b;
      float2 got;
      got.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
      got.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
      if (h) a = got;
      else b = got;
    }
}

__device__ __forceinline__ void line2_inverse(float2 (&v)[4][8], int h, const float2 *tw) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    dft_reg<float, 8, 1>(v[g]);
    const int n2 = 4 * h + g;
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) v[g][k1] = cmul<float>(v[g][k1], tw[n2 * k1]);
  }
  pair_exchange(v, h, false);
  // k1 = 4h + j: b[n2] = v[n2 % 4][4 (n2 / 4) + j]; outputs back into the same 8 slots
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 b[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) b[n2] = v[n2 & 3][4 * (n2 >> 2) + j];
    dft_reg<float, 8, 1>(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k2 & 3][4 * (k2 >> 2) + j] = b[k2];
  }
}

__device__ __forceinline__ void line2_forward(float2 (&v)[4][8], int h, const float2 *tw) {
  // k1 = 4h + j, values over k2 at v[k2 % 4][4 (k2 / 4) + j]: transform over k2 -> q2, twiddle
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 b[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) b[k2] = v[k2 & 3][4 * (k2 >> 2) + j];
    dft_reg<float, 8, -1>(b);
    const int k1 = 4 * h + j;
#pragma unroll
    for (int q2 = 0; q2 < 8; ++q2) v[q2 & 3][4 * (q2 >> 2) + j] = q2 == 0 ? b[q2] : cmulc<float>(b[q2], tw[k1 * q2]);
  }
  // lane h keeps q2 = 4h + g: it sends (k1 = 4h + j, q2 = 4(1-h) + g) from v[g][4(1-h) + j]
  pair_exchange(v, h, true);
  // q2 = 4h + g: a[k1] = v[g][k1]; transform over k1 -> q1; Y[4h + g + 8 q1] at v[g][q1]
#pragma unroll
  for (int g = 0; g < 4; ++g) dft_reg<float, 8, -1>(v[g]);
}

template <int N>
__global__ void __launch_bounds__(2 * N, 4) k_plane_reg2(Geo g, const float2 *__restrict__ twg, const int *__restrict__ jidx,
                                                      PlaneArgs<float> pa) {
  static_assert(N == 64, "two-thread lines are written for 64 = 8 x 8");
  constexpr int P = N + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 *tw = reinterpret_cast<float2 *>(smraw);
  float2 *tile = tw + N;
  float *vsm = reinterpret_cast<float *>(tile + N * P);
  int *xact = reinterpret_cast<int *>(vsm + N * P);
  const int t = threadIdx.x, z = blockIdx.y, q = blockIdx.x;
  const int line = t >> 1, h = t & 1;
  const int nx = g.nxact, xmax = g.xmax;
  if (t < N) tw[t] = twg[t];
  for (int i = t; i < nx; i += 2 * N) xact[i] = g.xactn[i];
  const float4 *vz = reinterpret_cast<const float4 *>(pa.field + (size_t)z * N * N);
  for (int i = t; i < N * N / 4; i += 2 * N) {  // 16-byte loads, padded rows
    const int row = i / (N / 4), c = 4 * (i % (N / 4));
    const float4 w = vz[i];
    vsm[row * P + c] = w.x;
    vsm[row * P + c + 1] = w.y;
    vsm[row * P + c + 2] = w.z;
    vsm[row * P + c + 3] = w.w;
  }
  __syncthreads();
  float2 *cbz = pa.cb + (size_t)q * g.n3 * g.ldcb + (size_t)z * g.ldcb;
  float2 v[4][8];
  const bool warp_cols = (t & ~31) / 2 < nx;  // some line of this warp is an occupied column
  if (warp_cols) {  // inverse along n2 of occupied column x (lanes of unoccupied lines run on zeros)
    const bool mine = line < nx;
    const int x = mine ? xact[line] : 0;
#pragma unroll
    for (int gg = 0; gg < 4; ++gg)
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) {
        const int y = 4 * h + gg + 8 * n1;
        const int jj = mine ? __ldg(jidx + y * N + x) : -1;
        v[gg][n1] = jj >= 0 ? cbz[jj] : make_float2(0.f, 0.f);
      }
    line2_inverse(v, h, tw);
    if (mine)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) tile[(4 * h + j + 8 * k2) * P + x] = v[k2 & 3][4 * (k2 >> 2) + j];
  }
  __syncthreads();
  {  // row y: inverse along n1, V_loc, forward along n1
    const int y = line;
#pragma unroll
    for (int gg = 0; gg < 4; ++gg)
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) {
        const int x = 4 * h + gg + 8 * n1;
        v[gg][n1] = (x <= xmax || x >= N - xmax) ? tile[y * P + x] : make_float2(0.f, 0.f);
      }
    line2_inverse(v, h, tw);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        float2 &e = v[k2 & 3][4 * (k2 >> 2) + j];
        e = cscal<float>(e, vsm[y * P + 4 * h + j + 8 * k2]);
      }
    line2_forward(v, h, tw);
#pragma unroll
    for (int gg = 0; gg < 4; ++gg)
#pragma unroll
      for (int q1 = 0; q1 < 8; ++q1) {
        const int x = 4 * h + gg + 8 * q1;
        if (x <= xmax || x >= N - xmax) tile[y * P + x] = v[gg][q1];
      }
  }
  __syncthreads();
  if (warp_cols) {  // forward along n2 of occupied column x, scattered back to the column buffer
    const bool mine = line < nx;
    const int x = mine ? xact[line] : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2)
        v[k2 & 3][4 * (k2 >> 2) + j] = mine ? tile[(4 * h + j + 8 * k2) * P + x] : make_float2(0.f, 0.f);
    line2_forward(v, h, tw);
    if (mine)
#pragma unroll
      for (int gg = 0; gg < 4; ++gg)
#pragma unroll
        for (int q1 = 0; q1 < 8; ++q1) {
          const int y = 4 * h + gg + 8 * q1;
          const int jj = __ldg(jidx + y * N + x);
          if (jj >= 0) cbz[jj] = v[gg][q1];
        }
  }
}

// sizes with the register kernels: N = 8 R2, R2 in {3, 4, 5, 8}
#define WDF_REG_SIZES(X) X(24) X(32) X(40) X(64)

static bool reg_plane_enabled() {
  static const bool on = std::getenv("WDF_NO_REG_PLANE") == nullptr;
  return on;
}

template <int N> size_t reg_smem(const Geo &g) {
  return sizeof(float2) * ((size_t)N + (size_t)N * (N + 1)) + sizeof(float) * (size_t)N * (N + 1) + sizeof(int) * (size_t)g.nxact;
}

template <int N> static void launch_reg(const FftCtx<float> &f, int nblk, const PlaneArgs<float> &pa, cudaStream_t st) {
  launch("plane_vloc", 32, k_plane_reg<N>, dim3(nblk, f.g.n3), dim3(N), reg_smem<N>(f.g), st, f.g, f.tw1, f.jidx, pa);
  WDF_CUDA_TRY(cudaGetLastError());
}


void set_plane_reg_limits(const Geo &g) {
  if (g.n1 == 64) raise_smem_limit(k_plane_reg2<64>, reg_smem<64>(g));
  switch (g.n1) {
#define X(N)                                                                                                   \
  case N:                                                                                                      \
    raise_smem_limit(k_plane_reg<N>, (size_t)((int)reg_smem<N>(g))); \
    break;
    WDF_REG_SIZES(X)
#undef X
    default: break;
  }
}

static bool launch_plane_reg2(const FftCtx<float> &f, int nblk, const PlaneArgs<float> &pa, cudaStream_t st) {
  if (f.g.n1 != 64 || f.g.n2 != 64) return false;
  launch("plane_vloc", 32, k_plane_reg2<64>, dim3(nblk, f.g.n3), dim3(128), reg_smem<64>(f.g), st, f.g, f.tw1, f.jidx, pa);
  WDF_CUDA_TRY(cudaGetLastError());
  return true;
}

static bool launch_plane_reg(const FftCtx<float> &f, int nblk, const PlaneArgs<float> &pa, cudaStream_t st) {
  if (!reg_plane_enabled() || f.g.n1 != f.g.n2) return false;
  switch (f.g.n1) {
#define X(N) \
  case N: launch_reg<N>(f, nblk, pa, st); return true;
    WDF_REG_SIZES(X)
#undef X
    default: return false;
  }
}

template <typename T, int N> size_t fast_smem(const Geo &g) {
  return sizeof(cplx<T>) * ((size_t)N + (size_t)N * (N + 1)) + sizeof(int) * (size_t)g.nxact;
}

template <typename T, int N> static void set_limits(const Geo &g) {
  const int sm = (int)fast_smem<T, N>(g);
  raise_smem_limit(k_plane_fast<T, N, OP_VLOC>, (size_t)(sm));
  raise_smem_limit(k_plane_fast<T, N, OP_G2R>, (size_t)(sm));
  raise_smem_limit(k_plane_fast<T, N, OP_PROD_R2G>, (size_t)(sm));
}

template <typename T, int N>
static void launch_n(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st) {
  dim3 grid(nblk, f.g.n3);
  const size_t sm = fast_smem<T, N>(f.g);
  constexpr int TH = PlaneShape<N>::threads;
  switch (op) {
    case OP_VLOC: launch("plane_vloc", bits_of<T>(), k_plane_fast<T, N, OP_VLOC>, grid, dim3(TH), sm, st, f.g, f.tw1, f.jidx, pa); break;
    case OP_G2R: launch("plane_g2r", bits_of<T>(), k_plane_fast<T, N, OP_G2R>, grid, dim3(TH), sm, st, f.g, f.tw1, f.jidx, pa); break;
    case OP_PROD_R2G:
      launch("plane_prod", bits_of<T>(), k_plane_fast<T, N, OP_PROD_R2G>, grid, dim3(TH), sm, st, f.g, f.tw1, f.jidx, pa);
      break;
    default: break;
  }
  WDF_CUDA_TRY(cudaGetLastError());
}

// sizes with a specialised kernel (n1 = n2 = N, FP64 tiles must fit 227 KB of shared memory)
#define WDF_FAST_SIZES(X) X(24) X(30) X(32) X(48) X(64) X(96)

bool plane_fast_supported(int n1, int n2) {
  if (n1 != n2) return false;
  switch (n1) {
#define X(N) case N:
    WDF_FAST_SIZES(X)
#undef X
    return true;
    default: return false;
  }
}

template <typename T> void set_plane_fast_limits(const Geo &g) {
  if (std::is_same<T, float>::value && g.n1 == g.n2) {
    set_plane_reg_limits(g);
    set_plane_pipe_limits(g);
  }
  if (std::is_same<T, df64>::value) set_plane_df_limits(g);
  switch (g.n1) {
#define X(N) \
  case N: set_limits<T, N>(g); break;
    WDF_FAST_SIZES(X)
#undef X
    default: break;
  }
}

template <typename T> bool launch_plane_fast(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st) {
  // the orbital sum of the density response keeps two register blocks across its loop and
  // spills here; it runs once per chi0 application and stays on the generic kernel
  const int v = op == OP_VLOC ? f.vloc_variant : 0;  // chosen at setup by timing (0: this order)
  if constexpr (std::is_same<T, df64>::value) {
    // the double-float 64 x 64 kernel: V_loc when the setup timing chose it, the product and the
    // orbital sum whenever it exists
    const bool use = op == OP_VLOC ? v == 6 : (op == OP_PROD_R2G || op == OP_ACCUM);
    if (use && launch_plane_df(f, op, nblk, pa, st)) return true;
  }
  if (op == OP_ACCUM || f.jidx == nullptr) return false;
  if (v == 3) return false;
  if constexpr (std::is_same<T, float>::value) {
    if (op == OP_VLOC && v == 5 && launch_plane_pipe(f, nblk, pa, st)) return true;
    if (op == OP_VLOC && v == 4 && launch_plane_reg2(f, nblk, pa, st)) return true;
    if (op == OP_VLOC && v != 2 && launch_plane_reg(f, nblk, pa, st)) return true;
  }
  if (!plane_fast_supported(f.g.n1, f.g.n2)) return false;
  switch (f.g.n1) {
#define X(N) \
  case N: launch_n<T, N>(f, op, nblk, pa, st); return true;
    WDF_FAST_SIZES(X)
#undef X
    default: return false;
  }
}

template <typename T> bool plane_variant_available(const FftCtx<T> &f, int v) {
  const Geo &g = f.g;
  if (v == 3) return true;
  if (f.jidx == nullptr) return false;
  if (v == 4) return std::is_same<T, float>::value && reg_plane_enabled() && g.n1 == 64 && g.n2 == 64;
  if (v == 5) return std::is_same<T, float>::value && plane_pipe_available(g, f.err);
  if (v == 6) return std::is_same<T, df64>::value && plane_df_available(g, f.jidx);
  if (v == 2) return plane_fast_supported(g.n1, g.n2);
  if (v == 1 && std::is_same<T, float>::value && reg_plane_enabled() && g.n1 == g.n2) {
    switch (g.n1) {
#define X(N) \
  case N: return true;
      WDF_REG_SIZES(X)
#undef X
      default: return false;
    }
  }
  return false;
}
template bool plane_variant_available<double>(const FftCtx<double> &, int);
template bool plane_variant_available<float>(const FftCtx<float> &, int);
template bool plane_variant_available<df64>(const FftCtx<df64> &, int);

template void set_plane_fast_limits<double>(const Geo &);
template void set_plane_fast_limits<float>(const Geo &);
template void set_plane_fast_limits<df64>(const Geo &);
template bool launch_plane_fast<double>(const FftCtx<double> &, int, int, const PlaneArgs<double> &, cudaStream_t);
template bool launch_plane_fast<float>(const FftCtx<float> &, int, int, const PlaneArgs<float> &, cudaStream_t);
template bool launch_plane_fast<df64>(const FftCtx<df64> &, int, int, const PlaneArgs<df64> &, cudaStream_t);

}  // namespace wdf

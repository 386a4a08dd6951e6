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
//
// This header holds the kernel and its per-size launch helpers; plane_fast.cu instantiates the
// common sizes and plane_more_*.cu the further sizes of cubic cells at a fixed grid spacing (one
// translation unit per precision and size group, compiled in parallel).
#pragma once

#include <cstdlib>

#include "fft.cuh"
#include "kernels.cuh"
#include "stockham.cuh"

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

// dispatch over a list of sizes: the first size equal to n1 (= n2) handles the call
template <typename T, int... Ns> struct PlaneFastSizes {
  static bool supported(int n1, int n2) { return n1 == n2 && ((n1 == Ns) || ...); }
  static void limits(const Geo &g) { ((g.n1 == Ns ? set_limits<T, Ns>(g) : void()), ...); }
  static bool launch(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st) {
    if (f.g.n1 != f.g.n2) return false;
    return ((f.g.n1 == Ns ? (launch_n<T, Ns>(f, op, nblk, pa, st), true) : false) || ...);
  }
};

}  // namespace wdf

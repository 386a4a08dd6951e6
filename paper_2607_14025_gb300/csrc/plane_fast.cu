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

#include "plane_fast_impl.cuh"
#include "plane_reg.cuh"

namespace wdf {

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

// sizes with a specialised kernel (n1 = n2 = N, FP64 tiles must fit 227 KB of shared memory)
#define WDF_FAST_SIZES(X) X(24) X(30) X(32) X(48) X(64) X(96)

// further sizes (plane_more_*.cu; float and double-float only)
#define WDF_MORE_SIZES_DF_A 36, 40, 45, 50, 54
#define WDF_MORE_SIZES_DF_B 60, 72, 75, 80
#define WDF_MORE_SIZES WDF_MORE_SIZES_DF_A, WDF_MORE_SIZES_DF_B
static bool plane_more_supported(int n1, int n2) { return PlaneFastSizes<float, WDF_MORE_SIZES>::supported(n1, n2); }

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
    set_plane_pipe2_limits(g);
  }
  if (std::is_same<T, df64>::value) set_plane_df_limits(g);
  if constexpr (std::is_same<T, float>::value) set_plane_more_limits_f32(g);
  if constexpr (std::is_same<T, df64>::value) {
    set_plane_more_limits_df_a(g);
    set_plane_more_limits_df_b(g);
  }
  switch (g.n1) {
#define X(N) \
  case N: set_limits<T, N>(g); break;
    WDF_FAST_SIZES(X)
#undef X
    default: break;
  }
}

template <typename T> bool launch_plane_fast(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st) {
  const int v = op == OP_VLOC ? f.vloc_variant : 0;  // chosen at setup by timing (0: this order)
  if constexpr (std::is_same<T, df64>::value) {
    // the double-float 64 x 64 kernel: V_loc when the setup timing chose it, the product and the
    // orbital sum whenever it exists
    const bool use = op == OP_VLOC ? v == 6 : (op == OP_PROD_R2G || op == OP_ACCUM);
    if (use && launch_plane_df(f, op, nblk, pa, st)) return true;
  }
  // the orbital sum of the density response keeps two register blocks across its loop and
  // spills in the Stockham kernel; it runs once per chi0 application and, outside the 64 x 64
  // double-float kernel above, stays on the generic kernel
  if (op == OP_ACCUM || f.jidx == nullptr) return false;
  if (v == 3) return false;
  // the other plane operations follow the setup timing of the V_loc product: where the generic
  // kernel won it (large double-float planes), they use the generic kernel too
  if (op != OP_VLOC && f.vloc_variant == 3) return false;
  if constexpr (std::is_same<T, float>::value) {
    if (op == OP_VLOC && v == 5 && launch_plane_pipe(f, nblk, pa, st)) return true;
    if (op == OP_VLOC && v == 7 && launch_plane_pipe2(f, nblk, pa, st)) return true;
    if (op == OP_VLOC && v == 4 && launch_plane_reg2(f, nblk, pa, st)) return true;
    if (op == OP_VLOC && v != 2 && launch_plane_reg(f, nblk, pa, st)) return true;
  }
  if (!plane_fast_supported(f.g.n1, f.g.n2)) {
    if constexpr (std::is_same<T, float>::value) return launch_plane_more_f32(f, op, nblk, pa, st);
    if constexpr (std::is_same<T, df64>::value) return launch_plane_more_df_a(f, op, nblk, pa, st) || launch_plane_more_df_b(f, op, nblk, pa, st);
    return false;
  }
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
  if (v == 7) return std::is_same<T, float>::value && plane_pipe2_available(g, f.err);
  if (v == 6) return std::is_same<T, df64>::value && plane_df_available(g, f.jidx);
  if (v == 2) return plane_fast_supported(g.n1, g.n2) || (!std::is_same<T, double>::value && plane_more_supported(g.n1, g.n2));
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
// the orbital sum of the density response as compile-time G2R transforms of each orbital's pair
// followed by a separate sum over orbitals (k_orbital_sum): FP64-class arithmetic on grids with a
// compile-time Stockham kernel, except the 64 x 64 double-float planes, whose kernel sums in place
template <typename T> bool plane_accum_by_g2r(const FftCtx<T> &f) {
  if constexpr (std::is_same<T, float>::value) {
    return false;
  } else {
    if (f.jidx == nullptr || f.vloc_variant == 3) return false;
    if constexpr (std::is_same<T, df64>::value)
      if (plane_df_available(f.g, f.jidx)) return false;
    return plane_fast_supported(f.g.n1, f.g.n2) || (!std::is_same<T, double>::value && plane_more_supported(f.g.n1, f.g.n2));
  }
}
template bool plane_accum_by_g2r<double>(const FftCtx<double> &);
template bool plane_accum_by_g2r<float>(const FftCtx<float> &);
template bool plane_accum_by_g2r<df64>(const FftCtx<df64> &);

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

// Dense linear algebra and conjugate-gradient kernels on blocks of plane-wave vectors.
//
// Vectors are rows of ld complex elements in the internal column layout; elements of column
// (0, 0) carry weight 1 in inner products and all others weight 2 (each stands for G and -G), so
// <a, b> = sum_e w_e Re(conj(a_e) b_e) is the inner product of the real functions. Padding
// elements are zero and stay zero. All reductions run in a fixed order (no floating-point
// atomics), so every result is bitwise reproducible.
#include <cfloat>

#include "kernels.cuh"

namespace wdf {

static __device__ __forceinline__ double wgt(int e, int len0) { return e < len0 ? 1.0 : 2.0; }

template <typename T> __device__ __forceinline__ double dre(cplx<T> a, cplx<T> b) {
  return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}
// per-thread partial sums of the inner CG: FP32 for FP32 vectors (a thread adds a few terms; the
// block reduction is FP64), FP64 otherwise. GB300 runs FP64 at 1/61 of the FP32 rate.
template <typename T> using PartAcc = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
template <typename T> __device__ __forceinline__ PartAcc<T> dre_acc(cplx<T> a, cplx<T> b) {
  typedef PartAcc<T> A;
  return (A)a.x * (A)b.x + (A)a.y * (A)b.y;
}

// Accumulators of the Gram and linear-combination kernels: a plain sum of products for FP64 (and
// FP32) elements; for double-float elements the lazy compensated sum DfAcc (12 FP32 operations a
// term instead of 18), renormalised every few terms.
template <typename A> struct AccOf {
  using type = A;
};
template <> struct AccOf<df64> {
  using type = DfAcc;
};
template <typename A> __device__ __forceinline__ void acc_zero(A &a) { a = 0; }
__device__ __forceinline__ void acc_zero(DfAcc &a) { a.s = a.c = 0.f; }
// a += x.x y.x + x.y y.y (the real part of conj(x) y)
template <typename A, typename C> __device__ __forceinline__ void acc_dre(A &a, C x, C y) {
  a += (A)x.x * (A)y.x + (A)x.y * (A)y.y;
}
__device__ __forceinline__ void acc_dre(DfAcc &a, cplx<df64> x, cplx<df64> y) {
  df_acc_fma(a, x.x, y.x);
  df_acc_fma(a, x.y, y.y);
}
template <typename A, typename B> __device__ __forceinline__ void acc_mac(A &a, B x, B y) { a += x * y; }
__device__ __forceinline__ void acc_mac(DfAcc &a, df64 x, df64 y) { df_acc_fma(a, x, y); }
template <typename A> __device__ __forceinline__ void acc_renorm(A &) {}
__device__ __forceinline__ void acc_renorm(DfAcc &a) { df_acc_renorm(a); }
template <typename A> __device__ __forceinline__ A acc_value(const A &a) { return a; }
__device__ __forceinline__ df64 acc_value(const DfAcc &a) { return df_acc_value(a); }

// block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024); result valid in
// thread 0
static __device__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// ---------------------------------------------------------------------------------------------
// Gram products out[i][j] = <A_i, B_j>

// Gram products: block tile GI x GJ = 64 x 128 outputs, 256 threads as 16 x 16, each thread a
// 4 x 8 register tile; element chunks of GK staged k-major in shared memory so that a thread
// reads 4 + 8 consecutive values per element (0.67 FMA per shared byte in FP32).
constexpr int GI = 64;
constexpr int GJ = 128;
constexpr int GK = 16;

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_gram(Geo g, const cplx<T> *__restrict__ A, int na, const cplx<T> *__restrict__ B,
                                             int nb, double *__restrict__ out, int ldo, int echunk, size_t split_stride) {
  __shared__ cplx<T> As[GK][GI];
  __shared__ cplx<T> Bs[GK][GJ];
  const int i0 = blockIdx.x * GI, j0 = blockIdx.y * GJ;
  const int ebeg = blockIdx.z * echunk;
  const int eend = min(g.nint, ebeg + echunk);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  typename AccOf<Acc>::type acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc_zero(acc[a][b]);
  for (int e0 = ebeg; e0 < eend; e0 += GK) {
    // 16 consecutive threads read 16 consecutive elements of one row
#pragma unroll
    for (int t = threadIdx.x; t < GI * GK; t += 256) {
      const int row = t / GK, col = t % GK, e = e0 + col;
      cplx<T> a = mkc<T>(0, 0);
      if (e < eend && i0 + row < na) {
        a = A[(size_t)(i0 + row) * g.ld + e];
        const T w = (T)wgt(e, g.len0);
        a = mkc<T>(a.x * w, a.y * w);
      }
      As[col][row] = a;
    }
#pragma unroll
    for (int t = threadIdx.x; t < GJ * GK; t += 256) {
      const int row = t / GK, col = t % GK, e = e0 + col;
      cplx<T> b = mkc<T>(0, 0);
      if (e < eend && j0 + row < nb) b = B[(size_t)(j0 + row) * g.ld + e];
      Bs[col][row] = b;
    }
    __syncthreads();
    for (int k0 = 0; k0 < GK; k0 += 4) {
#pragma unroll
      for (int k = k0; k < k0 + 4; ++k) {
        cplx<T> av[4], bv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 8; ++b) bv[b] = Bs[k][tx + 16 * b];  // consecutive lanes: consecutive banks
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc_dre(acc[a][b], av[a], bv[b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc_renorm(acc[a][b]);  // every 8 terms (double-float only)
    }
    __syncthreads();
  }
  double *o = out + blockIdx.z * split_stride;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx + 16 * b;
      if (i < na && j < nb) o[(size_t)i * ldo + j] = (double)acc_value(acc[a][b]);
    }
}

// FP32 Gram products: the same 64 x 128 block tile with 4 x 8 register tiles, 32-element chunks,
// and the next chunk's global loads issued before the current chunk's arithmetic (register
// prefetch), so memory latency overlaps the FMAs.
constexpr int GK32 = 32;

__global__ void __launch_bounds__(256) k_gram_f32(Geo g, const float2 *__restrict__ A, int na, const float2 *__restrict__ B, int nb,
                                                 double *__restrict__ out, int ldo, int echunk, size_t split_stride) {
  __shared__ float2 As[GK32][GI];
  __shared__ float2 Bs[GK32][GJ];
  const int i0 = blockIdx.x * GI, j0 = blockIdx.y * GJ;
  const int ebeg = blockIdx.z * echunk;
  const int eend = min(g.nint, ebeg + echunk);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  constexpr int LA = GI * GK32 / 256, LB = GJ * GK32 / 256;  // elements loaded per thread: 8, 16
  float2 ra[LA], rb[LB];
  auto load = [&](int e0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int t = threadIdx.x + 256 * u;
      const int row = t / GK32, col = t % GK32, e = e0 + col;
      float2 a = make_float2(0.f, 0.f);
      if (e < eend && i0 + row < na) {
        a = A[(size_t)(i0 + row) * g.ld + e];
        const float w = e < g.len0 ? 1.f : 2.f;
        a.x *= w;
        a.y *= w;
      }
      ra[u] = a;
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = threadIdx.x + 256 * u;
      const int row = t / GK32, col = t % GK32, e = e0 + col;
      rb[u] = (e < eend && j0 + row < nb) ? B[(size_t)(j0 + row) * g.ld + e] : make_float2(0.f, 0.f);
    }
  };
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  if (ebeg < eend) load(ebeg);
  for (int e0 = ebeg; e0 < eend; e0 += GK32) {
    __syncthreads();  // the previous chunk's arithmetic is done with the tiles
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int t = threadIdx.x + 256 * u;
      As[t % GK32][t / GK32] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = threadIdx.x + 256 * u;
      Bs[t % GK32][t / GK32] = rb[u];
    }
    __syncthreads();
    if (e0 + GK32 < eend) load(e0 + GK32);
#pragma unroll 8
    for (int k = 0; k < GK32; ++k) {
      float2 av[4], bv[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 8; ++b) bv[b] = Bs[k][tx + 16 * b];  // consecutive lanes: consecutive banks
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a].x, bv[b].x, fmaf(av[a].y, bv[b].y, acc[a][b]));
    }
  }
  double *o = out + blockIdx.z * split_stride;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx + 16 * b;
      if (i < na && j < nb) o[(size_t)i * ldo + j] = (double)acc[a][b];
    }
}

__global__ void k_sum_splits(const double *__restrict__ part, int nsplit, size_t stride, double *__restrict__ out, int na,
                             int nb, int ldo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= na * nb) return;
  const int i = t / nb, j = t % nb;
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += part[z * stride + (size_t)i * ldo + j];
  out[(size_t)i * ldo + j] = s;
}

// Gram products with at most 8 right-hand vectors (the Gram-Schmidt steps of the Davidson
// solver): one block per row of A computes all nb inner products; no wasted tile work.
constexpr int kNarrow = 8;

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_gram_narrow(Geo g, const cplx<T> *__restrict__ A, const cplx<T> *__restrict__ B, int nb,
                                                    double *__restrict__ out, int ldo) {
  const int i = blockIdx.x;
  Acc acc[kNarrow];
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) acc[j] = 0;
  const cplx<T> *a = A + (size_t)i * g.ld;
  for (int e = threadIdx.x; e < g.nint; e += blockDim.x) {
    const T w = (T)wgt(e, g.len0);
    const cplx<T> av = a[e];
    const Acc ax = (Acc)(av.x * w), ay = (Acc)(av.y * w);
#pragma unroll
    for (int j = 0; j < kNarrow; ++j)
      if (j < nb) {
        const cplx<T> bv = B[(size_t)j * g.ld + e];
        acc[j] += ax * (Acc)bv.x + ay * (Acc)bv.y;
      }
  }
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) {
    if (j >= nb) break;
    const double v = block_sum((double)acc[j]);
    if (threadIdx.x == 0) out[(size_t)i * ldo + j] = v;
  }
}

static int gram_nsplit(const Geo &g, int na, int nb, int &echunk) {
  const int tiles = ((na + GI - 1) / GI) * ((nb + GJ - 1) / GJ);
  int nsplit = 1;
  const int target = 4 * 2 * 152;  // four waves of two blocks per SM on the 152 SMs
  if (nb <= kNarrow) {
    echunk = g.nint;
    return 1;
  }
  if (tiles < target) nsplit = std::min(64, std::max(1, (target + tiles - 1) / tiles));
  echunk = (g.nint + nsplit - 1) / nsplit;
  echunk = ((echunk + GK - 1) / GK) * GK;
  return (g.nint + echunk - 1) / echunk;
}

size_t gram_work_doubles(const Geo &g, int na, int nb, int ldo) {
  int echunk;
  const int nsplit = gram_nsplit(g, na, nb, echunk);
  return nsplit > 1 ? (size_t)na * ldo * nsplit : 0;
}

// Split over elements when the output has too few tiles to fill the GPU; the partial sums go to
// work (caller-owned, gram_work_doubles() long) and are added in a fixed order.
template <typename T>
void launch_gram(const Geo &g, const cplx<T> *A, int na, const cplx<T> *B, int nb, double *out, int ldo, double *work,
                 size_t work_cap, cudaStream_t st) {
  if (na <= 0 || nb <= 0) return;
  typedef typename std::conditional<std::is_same<T, float>::value, float, T>::type AccN;
  if (nb <= kNarrow) {
    launch("gram", bits_of<T>(), k_gram_narrow<T, AccN>, dim3(na), dim3(256), 0, st, g, A, B, nb, out, ldo);
    WDF_CUDA_TRY(cudaGetLastError());
    return;
  }
  int echunk;
  int nsplit = gram_nsplit(g, na, nb, echunk);
  const size_t stride = (size_t)na * ldo;
  if (nsplit > 1 && (work == nullptr || work_cap < stride * nsplit)) {
    nsplit = 1;
    echunk = ((g.nint + GK - 1) / GK) * GK;
  }
  dim3 grid((na + GI - 1) / GI, (nb + GJ - 1) / GJ, nsplit);
  typedef typename std::conditional<std::is_same<T, float>::value, float, T>::type Acc;  // T for FP64 and double-float
  if constexpr (std::is_same<T, float>::value) {
    echunk = ((echunk + GK32 - 1) / GK32) * GK32;  // whole 32-element chunks per split
    grid.z = nsplit = (g.nint + echunk - 1) / echunk;
    if (nsplit == 1) {
      launch("gram", 32, k_gram_f32, dim3(grid), dim3(256), 0, st, g, A, na, B, nb, out, ldo, echunk, (size_t)0);
    } else {
      launch("gram", 32, k_gram_f32, dim3(grid), dim3(256), 0, st, g, A, na, B, nb, work, ldo, echunk, stride);
      WDF_CUDA_TRY(cudaGetLastError());
      launch("gram_sum", 0, k_sum_splits, dim3((na * nb + 255) / 256), dim3(256), 0, st, work, nsplit, stride, out, na, nb, ldo);
    }
    WDF_CUDA_TRY(cudaGetLastError());
    return;
  }
  if (nsplit == 1) {
    launch("gram", bits_of<T>(), k_gram<T, Acc>, dim3(grid), dim3(256), 0, st, g, A, na, B, nb, out, ldo, echunk, 0);
  } else {
    launch("gram", bits_of<T>(), k_gram<T, Acc>, dim3(grid), dim3(256), 0, st, g, A, na, B, nb, work, ldo, echunk, stride);
    WDF_CUDA_TRY(cudaGetLastError());
    launch("gram_sum", 0, k_sum_splits, dim3((na * nb + 255) / 256), dim3(256), 0, st, work, nsplit, stride, out, na, nb, ldo);
  }
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// linear combinations Y_s = c0 Y_s + sum_j U_j C[j][s] d_j

// Linear combinations: block tile LE x LS = 128 elements x 32 vectors; 256 threads, thread
// (te = tid % 32, ts = tid / 32) accumulates elements te + 32 p (p < 4, coalesced) of vectors
// 4 ts + q (q < 4). Rows of U and the scaled coefficients are staged LJ at a time; the
// coefficients a warp reads are one broadcast address.
constexpr int LE = 128;
constexpr int LS = 32;
template <typename T> __host__ __device__ constexpr int lj_rows() { return sizeof(T) == 8 ? 16 : 32; }  // 32 KB of U rows

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_lincomb(Geo g, cplx<T> *__restrict__ Y, int ny, const cplx<T> *__restrict__ U, int nu,
                                                const double *__restrict__ C, int ldc, const double *__restrict__ d, double c0,
                                                const cplx<T> *__restrict__ P, double *__restrict__ part) {
  constexpr int LJ = lj_rows<T>();
  __shared__ Acc cs[LJ][LS];
  __shared__ cplx<T> us[LJ][LE];
  const int te = threadIdx.x % 32, ts = threadIdx.x / 32;
  const int e0 = blockIdx.x * LE, s0 = blockIdx.y * LS;
  typename AccOf<Acc>::type ax[4][4], ay[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc_zero(ax[p][q]);
      acc_zero(ay[p][q]);
    }
  for (int j0 = 0; j0 < nu; j0 += LJ) {
    for (int t = threadIdx.x; t < LJ * LS; t += 256) {
      const int jj = t / LS, ss = t % LS;
      const int j = j0 + jj, s = s0 + ss;
      double v = 0.0;
      if (j < nu && s < ny) v = C[(size_t)j * ldc + s] * (d ? d[j] : 1.0);
      cs[jj][ss] = (Acc)v;
    }
    for (int t = threadIdx.x; t < LJ * LE; t += 256) {
      const int jj = t / LE, ee = t % LE;
      const int j = j0 + jj, e = e0 + ee;
      us[jj][ee] = (j < nu && e < g.nint) ? U[(size_t)j * g.ld + e] : mkc<T>(0, 0);
    }
    __syncthreads();
    const int jn = min(LJ, nu - j0);
    for (int jj = 0; jj < jn; ++jj) {
      cplx<T> u[4];
      Acc c[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) u[p] = us[jj][te + 32 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = cs[jj][ts * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc_mac(ax[p][q], c[q], (Acc)u[p].x);
          acc_mac(ay[p][q], c[q], (Acc)u[p].y);
        }
      if ((jj & 7) == 7 || jj == jn - 1) {  // renormalise every 8 terms (double-float only)
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc_renorm(ax[p][q]);
            acc_renorm(ay[p][q]);
          }
      }
    }
    __syncthreads();
  }
  typedef PartAcc<T> PA;
  PA dsum[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int s = s0 + ts * 4 + q;
    if (s >= ny) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = e0 + te + 32 * p;
      if (e >= g.nint) continue;
      cplx<T> *y = Y + (size_t)s * g.ld + e;
      cplx<T> yv;
      const Acc sx = acc_value(ax[p][q]), sy = acc_value(ay[p][q]);
      if (c0 == 0.0) {
        yv = mkc<T>((T)sx, (T)sy);
      } else {
        const cplx<T> o = *y;
        yv = mkc<T>((T)((Acc)c0 * (Acc)o.x + sx), (T)((Acc)c0 * (Acc)o.y + sy));
      }
      *y = yv;
      if (part) {  // partial inner products <P_s, Y_s> over this block's elements
        const cplx<T> pv = P[(size_t)s * g.ld + e];
        dsum[q] += (e < g.len0 ? (PA)1 : (PA)2) * dre_acc<T>(pv, yv);
      }
    }
  }
  if (part) {  // a warp holds vectors 4 ts .. 4 ts + 3 across its 32 lanes: reduce over lanes
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = (double)dsum[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      const int s = s0 + ts * 4 + q;
      if (te == 0 && s < ny) part[(size_t)s * gridDim.x + blockIdx.x] = v;
    }
  }
}

// Linear combinations into at most 8 vectors: each thread owns one element of every output.
template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_lincomb_narrow(Geo g, cplx<T> *__restrict__ Y, int ny, const cplx<T> *__restrict__ U, int nu,
                                                       const double *__restrict__ C, int ldc, const double *__restrict__ d, double c0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.nint) return;
  Acc ax[kNarrow], ay[kNarrow];
#pragma unroll
  for (int s = 0; s < kNarrow; ++s) ax[s] = ay[s] = 0;
  for (int j = 0; j < nu; ++j) {
    const cplx<T> u = U[(size_t)j * g.ld + e];
    const double dj = d ? d[j] : 1.0;
#pragma unroll
    for (int s = 0; s < kNarrow; ++s)
      if (s < ny) {
        const Acc c = (Acc)(C[(size_t)j * ldc + s] * dj);
        ax[s] += c * (Acc)u.x;
        ay[s] += c * (Acc)u.y;
      }
  }
#pragma unroll
  for (int s = 0; s < kNarrow; ++s) {
    if (s >= ny) break;
    cplx<T> *y = Y + (size_t)s * g.ld + e;
    if (c0 == 0.0) {
      *y = mkc<T>((T)ax[s], (T)ay[s]);
    } else {
      const cplx<T> o = *y;
      *y = mkc<T>((T)((Acc)c0 * (Acc)o.x + ax[s]), (T)((Acc)c0 * (Acc)o.y + ay[s]));
    }
  }
}

template <typename T>
void launch_lincomb(const Geo &g, cplx<T> *Y, int ny, const cplx<T> *U, int nu, const double *C, int ldc, const double *d,
                    double c0, cudaStream_t st) {
  if (ny <= 0) return;
  if (ny <= kNarrow) {
    typedef typename std::conditional<std::is_same<T, float>::value, float, T>::type AccN;
    launch("lincomb", bits_of<T>(), k_lincomb_narrow<T, AccN>, dim3((g.nint + 255) / 256), dim3(256), 0, st, g, Y, ny, U, nu, C, ldc,
           d, c0);
    WDF_CUDA_TRY(cudaGetLastError());
    return;
  }
  dim3 grid((g.nint + LE - 1) / LE, (ny + LS - 1) / LS);
  typedef typename std::conditional<std::is_same<T, float>::value, float, T>::type Acc;  // T for FP64 and double-float
  launch("lincomb", bits_of<T>(), k_lincomb<T, Acc>, dim3(grid), dim3(256), 0, st, g, Y, ny, U, nu, C, ldc, d, c0,
         (const cplx<T> *)nullptr, (double *)nullptr);
  WDF_CUDA_TRY(cudaGetLastError());
}

int lincomb_dot_chunks(const Geo &g) { return (g.nint + LE - 1) / LE; }

template <typename T>
bool launch_lincomb_dot(const Geo &g, cplx<T> *Y, int ny, const cplx<T> *U, int nu, const double *C, int ldc, const double *d,
                        double c0, const cplx<T> *P, double *part, cudaStream_t st) {
  if (ny <= kNarrow) return false;  // the narrow kernel has no dot epilogue
  dim3 grid((g.nint + LE - 1) / LE, (ny + LS - 1) / LS);
  typedef typename std::conditional<std::is_same<T, float>::value, float, T>::type Acc;
  launch("lincomb", bits_of<T>(), k_lincomb<T, Acc>, dim3(grid), dim3(256), 0, st, g, Y, ny, U, nu, C, ldc, d, c0, P, part);
  WDF_CUDA_TRY(cudaGetLastError());
  return true;
}

// ---------------------------------------------------------------------------------------------
// per-vector inner products in chunks

constexpr int DCHUNK = 2048;
int dot_chunks(const Geo &g) { return (g.nint + DCHUNK - 1) / DCHUNK; }

template <typename T>
__global__ void __launch_bounds__(256) k_dot_partial(Geo g, const cplx<T> *__restrict__ A, const cplx<T> *__restrict__ B,
                                                    double *__restrict__ part, int nchunk) {
  const int s = blockIdx.x, c = blockIdx.y;
  const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
  const cplx<T> *a = A + (size_t)s * g.ld, *b = B + (size_t)s * g.ld;
  double v = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) v += wgt(e, g.len0) * dre<T>(a[e], b[e]);
  v = block_sum(v);
  if (threadIdx.x == 0) part[(size_t)s * nchunk + c] = v;
}

template <typename T>
void launch_dot_partial(const Geo &g, const cplx<T> *A, const cplx<T> *B, int nvec, double *part, int nchunk, cudaStream_t st) {
  if (nvec <= 0) return;
  launch("dot_partial", bits_of<T>(), k_dot_partial<T>, dim3(dim3(nvec, nchunk)), dim3(256), 0, st, g, A, B, part, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

// per-vector partial sums of sum_e w_e |A_e - B_e|^2 with A in FP64 and B in FP32 (the deviation
// of an FP32 result from an FP64-class one), in the chunks of k_dot_partial
__global__ void __launch_bounds__(256) k_diff_partial(Geo g, const cplx<double> *__restrict__ A, const cplx<float> *__restrict__ B,
                                                     double *__restrict__ part, int nchunk) {
  const int s = blockIdx.x, c = blockIdx.y;
  const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
  const cplx<double> *a = A + (size_t)s * g.ld;
  const cplx<float> *b = B + (size_t)s * g.ld;
  double v = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double dx = a[e].x - (double)b[e].x, dy = a[e].y - (double)b[e].y;
    v += wgt(e, g.len0) * (dx * dx + dy * dy);
  }
  v = block_sum(v);
  if (threadIdx.x == 0) part[(size_t)s * nchunk + c] = v;
}

void launch_diff_partial(const Geo &g, const cplx<double> *A, const cplx<float> *B, int nvec, double *part, int nchunk, cudaStream_t st) {
  if (nvec <= 0) return;
  launch("dot_partial", 64, k_diff_partial, dim3(dim3(nvec, nchunk)), dim3(256), 0, st, g, A, B, part, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// conjugate gradients

template <typename T>
__global__ void __launch_bounds__(256) k_cg_start(Geo g, const cplx<T> *__restrict__ r, cplx<T> *z,
                                                 cplx<T> *__restrict__ p, const T *__restrict__ kprec, CgState s, int nchunk) {
  const int i = blockIdx.x, c = blockIdx.y;
  const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
  const size_t o = (size_t)i * g.ld;
  const T *K = kprec ? kprec + (size_t)s.vidx[i] * g.ld : nullptr;
  typedef PartAcc<T> A;
  A vrz = 0, vrr = 0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const cplx<T> rv = r[o + e];
    const T k = K ? K[e] : (T)1;
    const cplx<T> zv = mkc<T>(k * rv.x, k * rv.y);
    if (z) z[o + e] = zv;
    p[o + e] = zv;
    const A w = e < g.len0 ? (A)1 : (A)2;
    vrz += w * dre_acc<T>(rv, zv);
    vrr += w * dre_acc<T>(rv, rv);
  }
  const double brz = block_sum((double)vrz);
  const double brr = block_sum((double)vrr);
  if (threadIdx.x == 0) {
    s.part1[(size_t)i * nchunk + c] = brz;
    s.part2[(size_t)i * nchunk + c] = brr;
  }
}

template <typename T>
void launch_cg_start(const Geo &g, const cplx<T> *r, cplx<T> *z, cplx<T> *p, const T *kprec, const CgState &s, int n, int nchunk,
                     cudaStream_t st) {
  if (n <= 0) return;
  launch("cg_start", bits_of<T>(), k_cg_start<T>, dim3(dim3(n, nchunk)), dim3(256), 0, st, g, r, z, p, kprec, s, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(Geo g, cplx<T> *__restrict__ x, cplx<T> *__restrict__ r, cplx<T> *z,
                                                  const cplx<T> *__restrict__ p, const cplx<T> *__restrict__ Ap,
                                                  const T *__restrict__ kprec, CgState s, int nchunk) {
  const int i = blockIdx.x, c = blockIdx.y;
  typedef PartAcc<T> A;
  A vrz = 0, vrr = 0, vr3 = 0;
  // learned table: also <r, K_TPA r> while the solve is on its learned row (for a restart)
  const bool fb = s.krow && s.krow[i] < s.nocc;
  if (s.active[i]) {
    const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
    const size_t o = (size_t)i * g.ld, ox = (size_t)(s.home ? s.home[i] : i) * g.ld;
    const T *K = kprec ? kprec + (size_t)s.vidx[i] * g.ld : nullptr;
    const T *K3 = fb ? kprec + (size_t)(s.vorig[i] + s.nocc) * g.ld : nullptr;
    const T al = (T)(s.rz[i] / s.pap[i]);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const cplx<T> pv = p[o + e], av = Ap[o + e];
      cplx<T> xv = x[ox + e], rv = r[o + e];
      xv.x += al * pv.x;
      xv.y += al * pv.y;
      rv.x -= al * av.x;
      rv.y -= al * av.y;
      x[ox + e] = xv;
      r[o + e] = rv;
      const T k = K ? K[e] : (T)1;
      const cplx<T> zv = mkc<T>(k * rv.x, k * rv.y);
      if (z) z[o + e] = zv;  // z = K r is recomputed where needed when not stored
      const A w = e < g.len0 ? (A)1 : (A)2;
      const A rr = dre_acc<T>(rv, rv);
      vrz += w * dre_acc<T>(rv, zv);
      vrr += w * rr;
      if (K3) vr3 += w * (A)K3[e] * rr;
    }
  }
  const double brz = block_sum((double)vrz);
  const double brr = block_sum((double)vrr);
  const double br3 = fb ? block_sum((double)vr3) : 0.0;
  if (threadIdx.x == 0) {
    s.part1[(size_t)i * nchunk + c] = brz;
    s.part2[(size_t)i * nchunk + c] = brr;
    if (fb) s.part3[(size_t)i * nchunk + c] = br3;
  }
}

template <typename T>
void launch_cg_update(const Geo &g, cplx<T> *x, cplx<T> *r, cplx<T> *z, const cplx<T> *p, const cplx<T> *Ap, const T *kprec,
                      const CgState &s, int n, int nchunk, cudaStream_t st) {
  if (n <= 0) return;
  launch("cg_update", bits_of<T>(), k_cg_update<T>, dim3(dim3(n, nchunk)), dim3(256), 0, st, g, x, r, z, p, Ap, kprec, s, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void k_cg_direction(Geo g, cplx<T> *__restrict__ p, const cplx<T> *__restrict__ z, CgState s, int n) {
  const int i = blockIdx.x;
  if (!s.active[i]) return;
  const T be = (T)s.rz_new[i];  // holds beta after the scalar step
  const size_t o = (size_t)i * g.ld;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < g.nint; e += gridDim.y * blockDim.x) {
    const cplx<T> zv = z[o + e], pv = p[o + e];
    p[o + e] = mkc<T>(zv.x + be * pv.x, zv.y + be * pv.y);
  }
}

template <typename T>
void launch_cg_direction(const Geo &g, cplx<T> *p, const cplx<T> *z, const CgState &s, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int by = std::min(64, (g.nint + 255) / 256);
  launch("cg_direction", bits_of<T>(), k_cg_direction<T>, dim3(dim3(n, by)), dim3(256), 0, st, g, p, z, s, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

__global__ void k_cg_scalars(CgState s, int n, int nchunk, int which, int maxiter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0, b = 0.0;
  for (int c = 0; c < nchunk; ++c) a += s.part1[(size_t)i * nchunk + c];
  if (which != 0)
    for (int c = 0; c < nchunk; ++c) b += s.part2[(size_t)i * nchunk + c];
  if (which == 0) {
    s.pap[i] = a;
    if (s.active[i] && !(a > 0.0)) s.active[i] = 0;  // breakdown: keep the current iterate
    return;
  }
  if (which == 2) {  // start: r = b - A x0, z = K r
    s.rz[i] = a;
    s.rr[i] = b;
    const int act = (b > s.thr[i]) && (b > 0.0) && (s.iters[i] < maxiter);
    s.active[i] = act;
    if (act) atomicAdd(s.nactive, 1);
    if (s.krow) {
      s.rr_ref[i] = b;
      s.it_ref[i] = s.iters[i];
    }
    return;
  }
  if (!s.active[i]) return;
  s.iters[i] += 1;
  s.rr[i] = b;
  const double beta = a / s.rz[i];
  s.rz[i] = a;
  s.rz_new[i] = beta;
  if (b <= s.thr[i] || s.iters[i] >= maxiter || !(b == b)) {
    s.active[i] = 0;
    return;
  }
  atomicAdd(s.nactive, 1);
  if (s.krow && s.krow[i] < s.nocc && s.iters[i] - s.it_ref[i] >= 5) {
    if (b > 0.81 * s.rr_ref[i]) {  // stalled on the learned row: TPA from the current iterate
      double c3 = 0.0;
      for (int c = 0; c < nchunk; ++c) c3 += s.part3[(size_t)i * nchunk + c];
      s.krow[i] = s.vorig[i] + s.nocc;
      s.rz[i] = c3;
      s.rz_new[i] = 0.0;  // beta = 0: p = K_TPA r
      atomicAdd(s.nfb, 1);
    }
    s.rr_ref[i] = b;
    s.it_ref[i] = s.iters[i];
  }
}

void launch_cg_scalars(const CgState &s, int n, int nchunk, int which, int maxiter, cudaStream_t st) {
  if (n <= 0) return;
  launch("cg_scalars", 0, k_cg_scalars, dim3((n + 127) / 128), dim3(128), 0, st, s, n, nchunk, which, maxiter);
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// elementwise helpers

template <typename T>
__global__ void k_axpby(Geo g, cplx<T> *__restrict__ y, const cplx<T> *__restrict__ x, int n, double a, double b) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const cplx<T> xv = x[t];
    cplx<T> yv = y[t];
    if (b == 0.0) yv = mkc<T>(0, 0);
    y[t] = mkc<T>((T)(a * xv.x + b * yv.x), (T)(a * xv.y + b * yv.y));
  }
}
template <typename T> void launch_axpby(const Geo &g, cplx<T> *y, const cplx<T> *x, int n, double a, double b, cudaStream_t st) {
  if (n <= 0) return;
  launch("axpby", bits_of<T>(), k_axpby<T>, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, y, x, n, a, b);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void k_scale_rows(Geo g, cplx<T> *__restrict__ y, const double *__restrict__ coef, int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const T c = (T)coef[t / g.ld];
    y[t] = cscal<T>(y[t], c);
  }
}
template <typename T> void launch_scale_rows(const Geo &g, cplx<T> *y, const double *coef, int n, cudaStream_t st) {
  if (n <= 0) return;
  launch("scale_rows", bits_of<T>(), k_scale_rows<T>, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, y, coef, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename Tin, typename Tout>
__global__ void k_convert(Tout *__restrict__ y, const Tin *__restrict__ x, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) y[t] = (Tout)x[t];
}
// the orbital sum of the density response on the grid: acc = sum_v psi_v(r) G2R(dpsi_v pair)(r),
// the orbitals in ascending order (the same order as the in-plane sums)
template <typename R>
__global__ void k_orbital_sum(const cplx<R> *__restrict__ fields, const R *__restrict__ psir, int nocc, size_t ngrid,
                              cplx<R> *__restrict__ acc) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ngrid; i += (size_t)gridDim.x * blockDim.x) {
    cplx<R> a = cscal<R>(fields[i], psir[i]);
    for (int v = 1; v < nocc; ++v) a = cadd<R>(a, cscal<R>(fields[(size_t)v * ngrid + i], psir[(size_t)v * ngrid + i]));
    acc[i] = a;
  }
}

template <typename R>
void launch_orbital_sum(const cplx<R> *fields, const R *psir, int nocc, size_t ngrid, cplx<R> *acc, cudaStream_t st) {
  if (nocc <= 0) return;
  launch("orbital_sum", bits_of<R>(), k_orbital_sum<R>, dim3((int)std::min<size_t>(8192, (ngrid + 255) / 256)), dim3(256), 0, st, fields,
         psir, nocc, ngrid, acc);
  WDF_CUDA_TRY(cudaGetLastError());
}
template void launch_orbital_sum<double>(const cplx<double> *, const double *, int, size_t, cplx<double> *, cudaStream_t);
template void launch_orbital_sum<df64>(const cplx<df64> *, const df64 *, int, size_t, cplx<df64> *, cudaStream_t);

template <typename R> __global__ void k_fill(R *__restrict__ x, size_t count, R value) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) x[i] = value;
}
template <typename R> void launch_fill(R *x, size_t count, double value, cudaStream_t st) {
  launch("fill", bits_of<R>(), k_fill<R>, dim3((int)std::min<size_t>(8192, (count + 255) / 256)), dim3(256), 0, st, x, count, R(value));
  WDF_CUDA_TRY(cudaGetLastError());
}
template void launch_fill<double>(double *, size_t, double, cudaStream_t);
template void launch_fill<df64>(df64 *, size_t, double, cudaStream_t);

template <typename Tin, typename Tout> void launch_convert(const Geo &, Tout *y, const Tin *x, size_t count, cudaStream_t st) {
  if (count == 0) return;
  launch("convert", bits_of<Tout>(), k_convert<Tin, Tout>, dim3((int)std::min<size_t>(8192, (count + 255) / 256)), dim3(256), 0, st, y, x, count);
  WDF_CUDA_TRY(cudaGetLastError());
}

__global__ void k_ext_to_int(const double *__restrict__ ext, int n, int npw_h, const int *__restrict__ emap,
                             const int *__restrict__ emap2, const int *__restrict__ econj, const double *__restrict__ scale,
                             cplx<double> *__restrict__ out, int ld) {
  const size_t tot = (size_t)n * npw_h;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / npw_h), i = (int)(t % npw_h);
    double re = ext[2 * t], im = ext[2 * t + 1];
    const int e = emap[i];
    if (i == 0) im = 0.0;  // G = 0 coefficient of a real function is real
    if (econj[i]) im = -im;
    const double sc = scale ? scale[e] : 1.0;
    out[(size_t)s * ld + e] = mkc<double>(sc * re, sc * im);
    const int e2 = emap2[i];
    if (e2 >= 0) out[(size_t)s * ld + e2] = mkc<double>(sc * re, -sc * im);
  }
}
void launch_ext_to_int(const double *ext, int n, int npw_h, const int *emap, const int *emap2, const int *econj,
                       const double *scale_int, cplx<double> *out, int ld, cudaStream_t st) {
  if (n <= 0) return;
  const size_t tot = (size_t)n * npw_h;
  launch("ext_to_int", 0, k_ext_to_int, dim3((int)std::min<size_t>(8192, (tot + 255) / 256)), dim3(256), 0, st, ext, n, npw_h, emap, emap2, econj, scale_int, out, ld);
  WDF_CUDA_TRY(cudaGetLastError());
}

__global__ void k_int_to_ext(const cplx<double> *__restrict__ in, int n, int ld, int npw_h, const int *__restrict__ emap,
                             const int *__restrict__ econj, double *__restrict__ ext) {
  const size_t tot = (size_t)n * npw_h;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / npw_h), i = (int)(t % npw_h);
    const cplx<double> v = in[(size_t)s * ld + emap[i]];
    ext[2 * t] = v.x;
    ext[2 * t + 1] = (i == 0) ? 0.0 : (econj[i] ? -v.y : v.y);
  }
}
void launch_int_to_ext(const cplx<double> *in, int n, int ld, int npw_h, const int *emap, const int *econj, double *ext,
                       cudaStream_t st) {
  if (n <= 0) return;
  const size_t tot = (size_t)n * npw_h;
  launch("int_to_ext", 0, k_int_to_ext, dim3((int)std::min<size_t>(8192, (tot + 255) / 256)), dim3(256), 0, st, in, n, ld, npw_h, emap, econj, ext);
  WDF_CUDA_TRY(cudaGetLastError());
}

__global__ void k_ritz_residual(Geo g, cplx<double> *__restrict__ R, const cplx<double> *__restrict__ AX,
                                const cplx<double> *__restrict__ X, const double *__restrict__ theta, int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const double th = theta[t / g.ld];
    const cplx<double> a = AX[t], x = X[t];
    R[t] = mkc<double>(a.x - th * x.x, a.y - th * x.y);
  }
}
void launch_ritz_residual(const Geo &g, cplx<double> *R, const cplx<double> *AX, const cplx<double> *X, const double *theta, int n,
                          cudaStream_t st) {
  if (n <= 0) return;
  launch("ritz_residual", 0, k_ritz_residual, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, R, AX, X, theta, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

// Teter-Payne-Allan: K(x) = P / (P + 16 x^4), P = 27 + 18 x + 12 x^2 + 8 x^3, x = (|G|^2 / 2) / T_v
template <typename T>
__global__ void k_tpa_table(Geo g, T *__restrict__ K, const double *__restrict__ tkin, int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(t / g.ld), e = (int)(t % g.ld);
    double k = 0.0;
    if (e < g.nint) {
      const double x = 0.5 * g.g2[e] / tkin[v];
      const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
      k = p / (p + 16.0 * x * x * x * x);
    }
    K[t] = (T)k;
  }
}
template <typename T> void launch_tpa_table(const Geo &g, T *K, const double *tkin, int n, cudaStream_t st) {
  if (n <= 0) return;
  launch("tpa_table", bits_of<T>(), k_tpa_table<T>, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, K, tkin, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

// kinetic energy T_v = <x_v| -1/2 nabla^2 |x_v>, floored at 1e-3 hartree (a constant orbital would
// otherwise give a zero denominator in the preconditioner; the floor only changes iteration counts)
__global__ void k_kinetic(Geo g, const cplx<double> *__restrict__ X, double *__restrict__ tkin) {
  const int s = blockIdx.x;
  double v = 0.0;
  for (int e = threadIdx.x; e < g.nint; e += blockDim.x) {
    const cplx<double> x = X[(size_t)s * g.ld + e];
    v += wgt(e, g.len0) * 0.5 * g.g2[e] * (x.x * x.x + x.y * x.y);
  }
  v = block_sum(v);
  if (threadIdx.x == 0) tkin[s] = v > 1e-3 ? v : 1e-3;
}
void launch_kinetic(const Geo &g, const cplx<double> *X, int n, double *tkin, cudaStream_t st) {
  if (n <= 0) return;
  launch("kinetic", 0, k_kinetic, dim3(n), dim3(256), 0, st, g, X, tkin);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void k_mul_table(Geo g, cplx<T> *__restrict__ y, const T *__restrict__ tab, int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x)
    y[t] = cscal<T>(y[t], tab[t]);
}
template <typename T> void launch_mul_table(const Geo &g, cplx<T> *y, const T *tab, int n, cudaStream_t st) {
  if (n <= 0) return;
  launch("mul_table", bits_of<T>(), k_mul_table<T>, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, y, tab, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void k_check_finite(const T *__restrict__ x, size_t count, int *flag) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[t])) atomicExch(flag, 1);
}
template <typename T> void launch_check_finite(const T *x, size_t count, int *flag, cudaStream_t st) {
  if (count == 0) return;
  launch("check_finite", bits_of<T>(), k_check_finite<T>, dim3((int)std::min<size_t>(4096, (count + 255) / 256)), dim3(256), 0, st, x, count, flag);
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// Jacobi eigensolver (cyclic, parallel "round robin" ordering, two-sided rotations; Golub and
// Van Loan, Matrix Computations, Sec. 8.5). Each round rotates m/2 disjoint index pairs: one
// kernel rotates rows (and records cos/sin), one rotates columns of A and V.

static __device__ __forceinline__ void jac_pair(int m, int round, int i, int &p, int &q) {
  // circle method over players 0..m-1: player 0 fixed, the others rotate
  const int nm = m - 1;
  int a, b;
  if (i == 0) {
    a = 0;
    b = round % nm + 1;
  } else {
    a = (round + i) % nm + 1;
    b = (round - i + nm) % nm + 1;
  }
  p = min(a, b);
  q = max(a, b);
}

__global__ void k_jac_rows(double *__restrict__ A, int m, int round, double *__restrict__ cs, const int *__restrict__ done) {
  if (*done) return;
  int p, q;
  jac_pair(m, round, blockIdx.x, p, q);
  __shared__ double c_, s_;
  if (threadIdx.x == 0) {
    const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q], apq = A[(size_t)p * m + q];
    double c = 1.0, s = 0.0;
    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
      const double tau = (aqq - app) / (2.0 * apq);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      s = t * c;
    }
    c_ = c;
    s_ = s;
    cs[2 * blockIdx.x] = c;
    cs[2 * blockIdx.x + 1] = s;
  }
  __syncthreads();
  const double c = c_, s = s_;
  if (s == 0.0) return;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double ap = A[(size_t)p * m + k], aq = A[(size_t)q * m + k];
    A[(size_t)p * m + k] = c * ap - s * aq;
    A[(size_t)q * m + k] = s * ap + c * aq;
  }
}

__global__ void k_jac_cols(double *__restrict__ A, double *__restrict__ V, int m, int round, const double *__restrict__ cs,
                           const int *__restrict__ done) {
  if (*done) return;
  int p, q;
  jac_pair(m, round, blockIdx.x, p, q);
  const double c = cs[2 * blockIdx.x], s = cs[2 * blockIdx.x + 1];
  if (s == 0.0) return;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double ap = A[(size_t)k * m + p], aq = A[(size_t)k * m + q];
    A[(size_t)k * m + p] = c * ap - s * aq;
    A[(size_t)k * m + q] = s * ap + c * aq;
    const double vp = V[(size_t)k * m + p], vq = V[(size_t)k * m + q];
    V[(size_t)k * m + p] = c * vp - s * vq;
    V[(size_t)k * m + q] = s * vp + c * vq;
  }
}

__global__ void k_jac_init(const double *__restrict__ Ain, int n, double *__restrict__ A, double *__restrict__ V, int m, int *done) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
    const int i = t / m, j = t % m;
    double a = 0.0;
    if (i < n && j < n) a = 0.5 * (Ain[(size_t)i * n + j] + Ain[(size_t)j * n + i]);
    A[t] = a;
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0;
}

// converged when the off-diagonal Frobenius norm is below 1e-15 of the whole
__global__ void k_jac_check(const double *__restrict__ A, int m, int *done) {
  double off = 0.0, all = 0.0;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const double a = A[t];
    all += a * a;
    if (t / m != t % m) off += a * a;
  }
  off = block_sum(off);
  all = block_sum(all);
  if (threadIdx.x == 0 && off <= 1e-30 * all) *done = 1;
}

// sort eigenvalues ascending (ties by index) and copy out the first n
__global__ void k_jac_sort(const double *__restrict__ A, const double *__restrict__ Vw, int m, int n, double *__restrict__ w,
                           double *__restrict__ V) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = A[(size_t)i * m + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = A[(size_t)j * m + j];
      if (dj < di || (dj == di && j < i)) ++rank;
    }
    w[rank] = di;
    for (int k = 0; k < n; ++k) V[(size_t)k * n + rank] = Vw[(size_t)k * m + i];
  }
}

// Cholesky factorisation G = L L^T of an n x n symmetric positive definite matrix (FP64, one
// block, in shared memory) followed by the inverse of L; writes C[j * n + s] = (L^-1)[s][j] (so
// that Y_s = sum_j X_j C[j][s] is X L^-T) and sets *ok = 0 if a pivot falls below tol times the
// largest diagonal entry (near-dependent columns). Shared memory: L in the lower triangle, the
// strictly lower part of L^-1 transposed into the upper triangle, and the diagonal of L^-1 apart.
__global__ void k_chol_inv(const double *__restrict__ G, int n, double *__restrict__ C, double tol, int *ok) {
  extern __shared__ double sm[];
  double *A = sm;          // n x n
  double *dli = sm + n * n;  // diagonal of L^-1
  __shared__ double dmax;
  __shared__ int good;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    A[t] = (j <= i) ? 0.5 * (G[(size_t)i * n + j] + G[(size_t)j * n + i]) : 0.0;
  }
  if (threadIdx.x == 0) {
    good = 1;
    dmax = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < n; ++i) dmax = fmax(dmax, A[i * n + i]);
  __syncthreads();
  for (int j = 0; j < n; ++j) {  // right-looking: column j, then the trailing lower triangle
    if (threadIdx.x == 0) {
      const double d = A[j * n + j];
      if (!(d > tol * dmax)) good = 0;
      A[j * n + j] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double piv = A[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + j] /= piv;
    __syncthreads();
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = j + 1 + t / m, k = j + 1 + t % m;
      if (k <= i) A[i * n + k] -= A[i * n + j] * A[k * n + j];
    }
    __syncthreads();
  }
  // forward substitution L Li = I; thread c builds column c of Li: Li[c][c] -> dli[c],
  // Li[i][c] (i > c) -> A[c * n + i]
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    dli[c] = 1.0 / A[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double v = -A[i * n + c] * dli[c];
      for (int k = c + 1; k < i; ++k) v -= A[i * n + k] * A[c * n + k];
      A[c * n + i] = v / A[i * n + i];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int j = t / n, s2 = t % n;  // C[j][s] = Li[s][j]
    C[t] = (s2 < j) ? 0.0 : (s2 == j ? dli[j] : A[j * n + s2]);
  }
  if (threadIdx.x == 0) *ok = good;
}

size_t chol_inv_smem(int n) { return sizeof(double) * ((size_t)n * n + n); }

void launch_chol_inv(const double *G, int n, double *C, double tol, int *ok, cudaStream_t st) {
  launch("chol_inv", 0, k_chol_inv, dim3(1), dim3(256), chol_inv_smem(n), st, G, n, C, tol, ok);
  WDF_CUDA_TRY(cudaGetLastError());
}

void set_chol_inv_limits(int nmax) {
  raise_smem_limit(k_chol_inv, (size_t)((int)chol_inv_smem(nmax)));
}

// The whole eigensolve in one cooperative launch: block b of m/2 owns pair b of every round, a
// grid barrier separates the row rotations of a round from its column rotations and from the next
// round, and block 0 tests convergence after each sweep (the same rotations, order and test as
// the kernels above, without ~2 m launches per sweep). The barrier counts arrivals and bumps a
// generation number; a block waits for the bump with a bounded number of polls and, on expiry,
// sets the error flag and returns (the others then expire at their next barrier). Matrix entries
// written by other blocks are read past L1 (ld.global.cg), which is not coherent across SMs.
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, int *err, long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g0 = *(volatile unsigned *)gen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long it = 0;
      while (*(volatile unsigned *)gen == g0) {
        if (++it > limit) {
          ok = 0;
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// iw: [0] converged, [1] barrier arrivals, [2] barrier generation, [3] error
__global__ void __launch_bounds__(128) k_jac_coop(double *__restrict__ A, double *__restrict__ V, int m, int maxsweep, int *iw,
                                                  long limit) {
  const unsigned nb = gridDim.x;
  unsigned *count = reinterpret_cast<unsigned *>(iw + 1), *gen = reinterpret_cast<unsigned *>(iw + 2);
  int *err = iw + 3;
  __shared__ double c_, s_;
  __shared__ int stop;
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    for (int rd = 0; rd < m - 1; ++rd) {
      int p, q;
      jac_pair(m, rd, blockIdx.x, p, q);
      if (threadIdx.x == 0) {
        const double app = __ldcg(A + (size_t)p * m + p), aqq = __ldcg(A + (size_t)q * m + q), apq = __ldcg(A + (size_t)p * m + q);
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        c_ = c;
        s_ = s;
      }
      __syncthreads();
      const double c = c_, s = s_;
      if (s != 0.0)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
          const double ap = __ldcg(A + (size_t)p * m + k), aq = __ldcg(A + (size_t)q * m + k);
          __stcg(A + (size_t)p * m + k, c * ap - s * aq);
          __stcg(A + (size_t)q * m + k, s * ap + c * aq);
        }
      if (!grid_barrier(count, gen, nb, err, limit)) return;
      if (s != 0.0)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
          const double ap = __ldcg(A + (size_t)k * m + p), aq = __ldcg(A + (size_t)k * m + q);
          __stcg(A + (size_t)k * m + p, c * ap - s * aq);
          __stcg(A + (size_t)k * m + q, s * ap + c * aq);
          const double vp = __ldcg(V + (size_t)k * m + p), vq = __ldcg(V + (size_t)k * m + q);
          __stcg(V + (size_t)k * m + p, c * vp - s * vq);
          __stcg(V + (size_t)k * m + q, s * vp + c * vq);
        }
      if (!grid_barrier(count, gen, nb, err, limit)) return;
    }
    if (blockIdx.x == 0) {  // converged when the off-diagonal Frobenius norm is below 1e-15 of the whole
      double off = 0.0, all = 0.0;
      for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const double a = __ldcg(A + t);
        all += a * a;
        if (t / m != t % m) off += a * a;
      }
      off = block_sum(off);
      all = block_sum(all);
      if (threadIdx.x == 0) *(volatile int *)iw = off <= 1e-30 * all ? 1 : 0;
    }
    if (!grid_barrier(count, gen, nb, err, limit)) return;
    if (threadIdx.x == 0) stop = *(volatile int *)iw;
    __syncthreads();
    if (stop) break;
  }
}

// The eigensolve inside one cluster of kJacCl CTAs (m a multiple of 2 kJacCl, m <= 320): CTA c keeps
// rows [c R, (c + 1) R) of A and of V in its shared memory (R = m / kJacCl) and reaches the other
// CTAs' rows through distributed shared memory (mapa / ld,st.shared::cluster). Each round: the
// CTA that handles pair i (i mod kJacCl) computes (c, s) from A[p][p], A[q][q], A[p][q] and rotates
// rows p and q wherever they live; cluster barrier; every CTA rotates columns p and q of its own
// rows of A and V (local); cluster barrier. The hardware cluster barrier replaces the grid
// barrier's global atomics. Convergence: per-CTA partial sums, read by every CTA after a barrier,
// the same decision everywhere (the same test as the kernels above).
constexpr int kJacCl = 8;
constexpr int kJacThreads = 256;
constexpr int kJacMaxM = 320;

__device__ __forceinline__ uint32_t cl_addr(const void *local, uint32_t rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ double cl_ld(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st(uint32_t addr, double v) { asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory"); }
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared memory of one CTA: A rows [R][m], V rows [R][m], (c, s) of its pairs [m / 2][2] (entry i
// for the pairs i it handles), all pairs' (c, s) [m / 2][2], partial sums [2]
size_t jac_cluster_smem(int m) {
  const int R = m / kJacCl;
  return sizeof(double) * (2 * (size_t)R * m + 2 * (size_t)m + 2);
}

__global__ void __cluster_dims__(kJacCl, 1, 1) __launch_bounds__(kJacThreads)
    k_jac_cluster(double *__restrict__ Ag, double *__restrict__ Vg, int m, int maxsweep) {
  extern __shared__ __align__(16) double jsm[];
  const int R = m / kJacCl, np = m / 2;
  double *A = jsm, *V = A + (size_t)R * m, *csown = V + (size_t)R * m, *csall = csown + m, *part = csall + m;
  const uint32_t me = cl_rank();
  const int t = threadIdx.x, r0 = (int)me * R;
  for (int e = t; e < R * m; e += kJacThreads) {
    const int lr = e / m, k = e % m;
    A[e] = Ag[(size_t)(r0 + lr) * m + k];
    V[e] = (r0 + lr == k) ? 1.0 : 0.0;
  }
  cl_sync();  // every CTA's rows are in place before any remote access
  // the local address of row r of A in the CTA that owns it, as a cluster address
  auto arow = [&](int r) { return cl_addr(A + (size_t)(r % R) * m, (uint32_t)(r / R)); };
  const int ppc = np / kJacCl;             // pairs handled per CTA and round
  const int tpp = kJacThreads / ppc;       // threads per handled pair
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    for (int rd = 0; rd < m - 1; ++rd) {
      // rows: pair i = me + kJacCl * h (h < ppc), handled by threads [h tpp, (h + 1) tpp)
      {
        const int h = t / tpp, j = t % tpp, i = (int)me + kJacCl * h;
        const bool act = h < ppc;  // the threads past ppc tpp have no pair
        int p = 0, q = 1;
        if (act) jac_pair(m, rd, i, p, q);
        const uint32_t ap_row = arow(p), aq_row = arow(q);
        double app = 0.0, aqq = 0.0, apq = 0.0;
        if (act) {
          app = cl_ld(ap_row + 8u * p);
          aqq = cl_ld(aq_row + 8u * q);
          apq = cl_ld(ap_row + 8u * q);
        }
        double c = 1.0, s = 0.0;
        if (act && fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        if (act && j == 0) {
          csown[2 * i] = c;
          csown[2 * i + 1] = s;
        }
        __syncthreads();  // the pair's three entries are read before any of its threads rotates them
        if (act && s != 0.0)
          for (int k = j; k < m; k += tpp) {
            const double ap = cl_ld(ap_row + 8u * k), aq = cl_ld(aq_row + 8u * k);
            cl_st(ap_row + 8u * k, c * ap - s * aq);
            cl_st(aq_row + 8u * k, s * ap + c * aq);
          }
      }
      cl_sync();
      // columns: every pair's (c, s) from the CTA that handled it, then the local rows
      for (int i = t; i < np; i += kJacThreads) {
        const uint32_t src = cl_addr(csown + 2 * i, (uint32_t)(i % kJacCl));
        csall[2 * i] = cl_ld(src);
        csall[2 * i + 1] = cl_ld(src + 8u);
      }
      __syncthreads();
      for (int w = t; w < R * np; w += kJacThreads) {
        const int lr = w / np, i = w % np;
        const double c = csall[2 * i], s = csall[2 * i + 1];
        if (s == 0.0) continue;
        int p, q;
        jac_pair(m, rd, i, p, q);
        double *ar = A + (size_t)lr * m, *vr = V + (size_t)lr * m;
        const double ap = ar[p], aq = ar[q];
        ar[p] = c * ap - s * aq;
        ar[q] = s * ap + c * aq;
        const double vp = vr[p], vq = vr[q];
        vr[p] = c * vp - s * vq;
        vr[q] = s * vp + c * vq;
      }
      cl_sync();  // columns done everywhere before the next round reads rows and (c, s)
    }
    // convergence: off-diagonal and total squares of the local rows, combined in every CTA
    double off = 0.0, all = 0.0;
    for (int e = t; e < R * m; e += kJacThreads) {
      const double a = A[e];
      all += a * a;
      if (r0 + e / m != e % m) off += a * a;
    }
    off = block_sum(off);
    all = block_sum(all);
    if (t == 0) {
      part[0] = off;
      part[1] = all;
    }
    cl_sync();
    __shared__ int stop;
    if (t == 0) {
      double o = 0.0, a = 0.0;
      for (int c = 0; c < kJacCl; ++c) {
        const uint32_t src = cl_addr(part, (uint32_t)c);
        o += cl_ld(src);
        a += cl_ld(src + 8u);
      }
      stop = o <= 1e-30 * a ? 1 : 0;
    }
    __syncthreads();
    const bool done = stop != 0;
    cl_sync();  // every CTA has read the partials before the next sweep overwrites them
    if (done) break;
  }
  for (int e = t; e < R * m; e += kJacThreads) {
    const int lr = e / m, k = e % m;
    Ag[(size_t)(r0 + lr) * m + k] = A[e];
    Vg[(size_t)(r0 + lr) * m + k] = V[e];
  }
  cl_sync();  // no CTA leaves while another may still read its shared memory
}

void set_jacobi_limits(int nmax) {
  const int m = ((std::max(2, nmax) + 2 * kJacCl - 1) / (2 * kJacCl)) * (2 * kJacCl);
  if (m <= kJacMaxM) raise_smem_limit(k_jac_cluster, jac_cluster_smem(m));
}

__global__ void k_jac_coop_init(int *iw) {
  iw[0] = 0;
  iw[1] = 0;
  iw[3] = 0;
}

// the eigensolver's dimension: n padded to a multiple of 2 kJacCl (zero rows and columns, which
// no rotation ever mixes in; the sort reads the first n only)
static int jac_dim(int n) { return ((std::max(2, n) + 2 * kJacCl - 1) / (2 * kJacCl)) * (2 * kJacCl); }

size_t jacobi_work_doubles(int n) {
  const int m = jac_dim(n);
  return 2 * (size_t)m * m + 2 * (size_t)m;
}

void jacobi_eigh(double *Ain, double *Vout, double *w, int n, double *work, int *iwork, cudaStream_t st, long wait_limit) {
  if (n <= 0) return;
  const int mm = jac_dim(n);
  double *A = work, *V = work + (size_t)mm * mm, *cs = V + (size_t)mm * mm;
  int *done = iwork;
  launch("jac_init", 0, k_jac_init, dim3(std::min(1024, (mm * mm + 255) / 256)), dim3(256), 0, st, Ain, n, A, V, mm, done);
  WDF_CUDA_TRY(cudaGetLastError());
  const int maxsweep = 40;
  // one cluster of CTAs with the matrix in distributed shared memory
  static const bool cluster_off = std::getenv("WDF_NO_CLUSTER_JACOBI") != nullptr;
  if (!cluster_off && mm <= kJacMaxM) {
    k_jac_cluster<<<kJacCl, kJacThreads, jac_cluster_smem(mm), st>>>(A, V, mm, maxsweep);
    if (cudaGetLastError() == cudaSuccess) {
      g_launches.fetch_add(1, std::memory_order_relaxed);
      launch("jac_sort", 0, k_jac_sort, dim3(1), dim3(256), 0, st, A, V, mm, n, w, Vout);
      WDF_CUDA_TRY(cudaGetLastError());
      return;
    }
  }
  // one cooperative launch when every block of the eigensolve can be resident at once
  static const bool coop_off = std::getenv("WDF_NO_COOP_JACOBI") != nullptr;
  int dev = 0, coop = 0, nsm = 0, per_sm = 0;
  if (!coop_off && cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jac_coop, 128, 0) == cudaSuccess && coop && mm / 2 <= nsm * per_sm) {
    launch("jac_init", 0, k_jac_coop_init, dim3(1), dim3(1), 0, st, done);
    int m_arg = mm, ms_arg = maxsweep;
    long lim_arg = wait_limit > 0 ? wait_limit : kGridBarrierPolls;
    void *args[] = {&A, &V, &m_arg, &ms_arg, &done, &lim_arg};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    WDF_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_jac_coop, dim3(mm / 2), dim3(128), args, 0, st));
    launch("jac_sort", 0, k_jac_sort, dim3(1), dim3(256), 0, st, A, V, mm, n, w, Vout);
    WDF_CUDA_TRY(cudaGetLastError());
    return;
  }
  int hdone = 0;
  for (int sweep = 0; sweep < maxsweep && !hdone; ++sweep) {
    for (int rd = 0; rd < mm - 1; ++rd) {
      launch("jac_rows", 0, k_jac_rows, dim3(mm / 2), dim3(128), 0, st, A, mm, rd, cs, done);
      launch("jac_cols", 0, k_jac_cols, dim3(mm / 2), dim3(128), 0, st, A, V, mm, rd, cs, done);
    }
    launch("jac_check", 0, k_jac_check, dim3(1), dim3(1024), 0, st, A, mm, done);
    WDF_CUDA_TRY(cudaGetLastError());
    if (sweep % 3 == 2) {
      WDF_CUDA_TRY(cudaMemcpyAsync(&hdone, done, sizeof(int), cudaMemcpyDeviceToHost, st));
      WDF_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  launch("jac_sort", 0, k_jac_sort, dim3(1), dim3(256), 0, st, A, V, mm, n, w, Vout);
  WDF_CUDA_TRY(cudaGetLastError());
}

#define WDF_INST(T)                                                                                                   \
  template void launch_gram<T>(const Geo &, const cplx<T> *, int, const cplx<T> *, int, double *, int, double *,      \
                               size_t, cudaStream_t);                                                             \
  template void launch_lincomb<T>(const Geo &, cplx<T> *, int, const cplx<T> *, int, const double *, int, const double *, \
                                  double, cudaStream_t);                                                              \
  template void launch_dot_partial<T>(const Geo &, const cplx<T> *, const cplx<T> *, int, double *, int, cudaStream_t); \
  template void launch_cg_start<T>(const Geo &, const cplx<T> *, cplx<T> *, cplx<T> *, const T *, const CgState &, int,  \
                                   int, cudaStream_t);                                                                \
  template void launch_cg_update<T>(const Geo &, cplx<T> *, cplx<T> *, cplx<T> *, const cplx<T> *, const cplx<T> *,     \
                                    const T *, const CgState &, int, int, cudaStream_t);                             \
  template void launch_cg_direction<T>(const Geo &, cplx<T> *, const cplx<T> *, const CgState &, int, cudaStream_t);   \
  template bool launch_lincomb_dot<T>(const Geo &, cplx<T> *, int, const cplx<T> *, int, const double *, int, const double *, \
                                      double, const cplx<T> *, double *, cudaStream_t);                              \
  template void launch_axpby<T>(const Geo &, cplx<T> *, const cplx<T> *, int, double, double, cudaStream_t);          \
  template void launch_scale_rows<T>(const Geo &, cplx<T> *, const double *, int, cudaStream_t);                      \
  template void launch_tpa_table<T>(const Geo &, T *, const double *, int, cudaStream_t);                            \
  template void launch_check_finite<T>(const T *, size_t, int *, cudaStream_t);                                  \
  template void launch_mul_table<T>(const Geo &, cplx<T> *, const T *, int, cudaStream_t);
WDF_INST(double)
WDF_INST(float)
#undef WDF_INST
template void launch_convert<double, float>(const Geo &, float *, const double *, size_t, cudaStream_t);
template void launch_convert<float, double>(const Geo &, double *, const float *, size_t, cudaStream_t);
template void launch_convert<double, df64>(const Geo &, df64 *, const double *, size_t, cudaStream_t);
template void launch_convert<df64, double>(const Geo &, double *, const df64 *, size_t, cudaStream_t);
template void launch_gram<df64>(const Geo &, const cplx<df64> *, int, const cplx<df64> *, int, double *, int, double *, size_t,
                                cudaStream_t);
template void launch_lincomb<df64>(const Geo &, cplx<df64> *, int, const cplx<df64> *, int, const double *, int, const double *,
                                   double, cudaStream_t);

}  // namespace wdf

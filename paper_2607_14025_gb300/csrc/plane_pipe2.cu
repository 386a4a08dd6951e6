// Persistent FP32 V_loc plane kernel with two threads per line, for N x N planes (N = 8 R with R
// even, N a multiple of 32) whose occupied columns are the full disk |n1|, |n2| <= XM: the 96 x 96
// planes of the precision configuration (XM = 22), where a whole line no longer fits one
// thread's registers.
//
// Per unit (one z plane of one Gamma pair) it does what the 64 x 64 persistent kernel does: the
// inverse n2 transform of the NX = 2 XM + 1 occupied columns, the inverse n1 transform of every
// row, the product with V_loc(r), the forward n1 transform and the forward n2 transform of the
// occupied columns back to the column buffer; slices of the column buffer move by bulk copies
// (three in flight), and the forward column phase of unit k overlaps the inverse column phase of
// unit k + 1 (the two halves of the block, two tiles).
//
// A line of N points is split over a pair of lanes by a four-step DFT, N = 8 R with n = n2 + R n1
// and k = k1 + 8 k2: lane h holds the inputs with n2 in [h R/2, (h + 1) R/2) (R/2 groups of 8),
// does the 8-point DFTs over n1 and the twiddles w^(n2 k1), swaps half of its values with its
// partner (one shuffle per value sent) so that it holds k1 in [4h, 4h + 4) for every n2, and
// finishes with R-point DFTs over n2 (prime-factor 3 x 4 for R = 12). The forward transform runs
// the same steps backwards and returns natural order, so the pointwise product between the two
// row transforms stays in registers. Inputs outside the disk are compile-time zeros for whole
// groups n1 (pruned from the 8-point DFTs), and outputs outside it are never computed.
// Every wait is bounded: a block whose copy does not complete sets the error flag, waits (again
// bounded) for the copies it has in flight and leaves.
#include <cstdlib>

#include "bulk.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "stockham.cuh"

namespace wdf {
namespace {

constexpr long kCopyWaitLimit = 1L << 24;

template <int N> struct Line2 {
  static constexpr int R = N / 8;  // second-stage radix
  static constexpr int H = R / 2;  // first-stage groups per lane
  static_assert(N % 8 == 0 && R % 2 == 0, "N = 8 R with R even");
};

// group n1 of the first stage lies outside the disk |x| <= XM for both lanes: n = n2 + R n1 with
// n2 in [0, R) stays inside (XM, N - XM)
template <int N, int XM> __device__ __forceinline__ constexpr bool group_off(int n1) {
  return Line2<N>::R * n1 > XM && Line2<N>::R * n1 + Line2<N>::R - 1 < N - XM;
}
template <int N, int XM> __device__ __forceinline__ bool on_disk(int x) { return x <= XM || x >= N - XM; }
template <int N, int XM> __device__ __forceinline__ int compact(int x) { return x <= XM ? x : x - (N - (2 * XM + 1)); }

// lanes 2i and 2i + 1: lane h keeps slots [g][4h + j] and trades slots [g][4(1 - h) + j]
template <int H> __device__ __forceinline__ void pair_swap(float2 (&v)[H][8], int h) {
#pragma unroll
  for (int g = 0; g < H; ++g)
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

// inverse DFT (w = exp(+2 pi i / N)) of a line split over a lane pair. In: x[n2 + R n1] with
// n2 = H h + g at v[g][n1]. Out: X[k1 + 8 k2] with k1 = 4 h + j at v[k2 % H][4 (k2 / H) + j].
template <int N> __device__ __forceinline__ void line2_inverse(float2 (&v)[Line2<N>::H][8], int h, const float2 *tw) {
  constexpr int R = Line2<N>::R, H = Line2<N>::H;
#pragma unroll
  for (int g = 0; g < H; ++g) {
    dft_reg<float, 8, 1>(v[g]);
    const int n2 = H * h + g;
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) v[g][k1] = cmul<float>(v[g][k1], tw[n2 * k1]);
  }
  pair_swap<H>(v, h);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 b[R];
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) b[n2] = v[n2 % H][4 * (n2 / H) + j];
    dft_reg<float, R, 1>(b);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) v[k2 % H][4 * (k2 / H) + j] = b[k2];
  }
}

// forward DFT (w^-1), the inverse's steps backwards: in the inverse's output layout, out
// Y[q2 + R q1] with q2 = H h + g at v[g][q1]
template <int N> __device__ __forceinline__ void line2_forward(float2 (&v)[Line2<N>::H][8], int h, const float2 *tw) {
  constexpr int R = Line2<N>::R, H = Line2<N>::H;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 b[R];
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) b[k2] = v[k2 % H][4 * (k2 / H) + j];
    dft_reg<float, R, -1>(b);
    const int k1 = 4 * h + j;
#pragma unroll
    for (int q2 = 0; q2 < R; ++q2) v[q2 % H][4 * (q2 / H) + j] = q2 == 0 ? b[0] : cmulc<float>(b[q2], tw[k1 * q2]);
  }
  pair_swap<H>(v, h);
#pragma unroll
  for (int g = 0; g < H; ++g) dft_reg<float, 8, -1>(v[g]);
}

// inverse n2 transform of compact column l (natural x): slice -> tile column l (natural rows);
// `live` false: the pair runs on zeros and stores nothing (its lanes still take part in shuffles)
template <int N, int XM>
__device__ __forceinline__ void column_inverse(const float2 *sl, const int *__restrict__ jidx, int l, bool live, int h, float2 *tile,
                                               const float2 *tw) {
  constexpr int H = Line2<N>::H, R = Line2<N>::R, NX = 2 * XM + 1;
  const int x = l <= XM ? l : l + (N - NX);
  float2 v[H][8];
#pragma unroll
  for (int g = 0; g < H; ++g)
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      v[g][n1] = make_float2(0.f, 0.f);
      if (!group_off<N, XM>(n1) && live) {
        const int y = H * h + g + R * n1;
        if (on_disk<N, XM>(y)) {
          const int jj = __ldg(jidx + y * N + x);
          if (jj >= 0) v[g][n1] = sl[jj];
        }
      }
    }
  line2_inverse<N>(v, h, tw);
  if (live)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) tile[(4 * h + j + 8 * k2) * NX + l] = v[k2 % H][4 * (k2 / H) + j];
}

// forward n2 transform of compact column l back into the slice (disk rows only)
template <int N, int XM>
__device__ __forceinline__ void column_forward(float2 *sl, const int *__restrict__ jidx, int l, bool live, int h, const float2 *tile,
                                               const float2 *tw) {
  constexpr int H = Line2<N>::H, R = Line2<N>::R, NX = 2 * XM + 1;
  const int x = l <= XM ? l : l + (N - NX);
  float2 v[H][8];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2)
      v[k2 % H][4 * (k2 / H) + j] = live ? tile[(4 * h + j + 8 * k2) * NX + l] : make_float2(0.f, 0.f);
  line2_forward<N>(v, h, tw);
  if (live)
#pragma unroll
    for (int g = 0; g < H; ++g)
#pragma unroll
      for (int q1 = 0; q1 < 8; ++q1) {
        if (group_off<N, XM>(q1)) continue;
        const int y = H * h + g + R * q1;
        if (on_disk<N, XM>(y)) {
          const int jj = __ldg(jidx + y * N + x);
          if (jj >= 0) sl[jj] = v[g][q1];
        }
      }
}

// row y of the tile: inverse n1 transform, V_loc(r) product, forward n1 transform
template <int N, int XM>
__device__ __forceinline__ void row_vloc(float2 *tile, int y, int h, const float *__restrict__ vrow, const float2 *tw) {
  constexpr int H = Line2<N>::H, R = Line2<N>::R, NX = 2 * XM + 1;
  float2 *tr = tile + y * NX;
  float2 v[H][8];
#pragma unroll
  for (int g = 0; g < H; ++g)
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      v[g][n1] = make_float2(0.f, 0.f);
      if (!group_off<N, XM>(n1)) {
        const int x = H * h + g + R * n1;
        if (on_disk<N, XM>(x)) v[g][n1] = tr[compact<N, XM>(x)];
      }
    }
  line2_inverse<N>(v, h, tw);
  // real-space point r = 4 h + j + 8 k2 sits at v[k2 % H][4 (k2 / H) + j]: four consecutive j
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) {
    const float4 w = __ldg(reinterpret_cast<const float4 *>(vrow + 8 * k2 + 4 * h));
    float2 *e = &v[k2 % H][4 * (k2 / H)];
    e[0] = cscal<float>(e[0], w.x);
    e[1] = cscal<float>(e[1], w.y);
    e[2] = cscal<float>(e[2], w.z);
    e[3] = cscal<float>(e[3], w.w);
  }
  line2_forward<N>(v, h, tw);
#pragma unroll
  for (int g = 0; g < H; ++g)
#pragma unroll
    for (int q1 = 0; q1 < 8; ++q1) {
      if (group_off<N, XM>(q1)) continue;
      const int x = H * h + g + R * q1;
      if (on_disk<N, XM>(x)) tr[compact<N, XM>(x)] = v[g][q1];
    }
}

// threads: two per row; in the column phases the first half of the block (N threads, whole
// warps) runs the forward columns of one unit while the second half runs the inverse columns of
// the next
template <int N, int XM>
__global__ void __launch_bounds__(2 * N, 2) k_plane_pipe2(Geo g, const float2 *__restrict__ twg, const int *__restrict__ jidx,
                                                          PlaneArgs<float> pa, long nunits, int *err) {
  constexpr int NX = 2 * XM + 1;
  static_assert(N % 32 == 0, "each column phase takes whole warps");
  static_assert(2 * NX <= N, "a lane pair per occupied column in half the block");
  extern __shared__ __align__(128) unsigned char smraw[];
  const int ldcb = g.ldcb;
  float2 *slices = reinterpret_cast<float2 *>(smraw);  // 3 x ldcb
  float2 *tiles = slices + 3 * ldcb;                     // 2 x N x NX
  float2 *tw = tiles + 2 * N * NX;                       // N
  uint64_t *bar = reinterpret_cast<uint64_t *>(tw + N);  // 3
  const int t = threadIdx.x, h = t & 1, half = t / N, l = (t % N) >> 1;
  const bool live = l < NX;
  const long G = gridDim.x, u0 = blockIdx.x;
  if (u0 >= nunits) return;
  const int cnt = (int)((nunits - 1 - u0) / G) + 1;
  const uint32_t bytes = (uint32_t)ldcb * (uint32_t)sizeof(float2);
  float2 *cb = pa.cb;
  int issued[3] = {0, 0, 0};  // loads issued into each slice (thread 0)
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bar[i], 1);
    tc::fence_mbar_init();
  }
  if (t < N) tw[t] = twg[t];
  __syncthreads();
  if (t == 0) {
    bulk::load(slices, cb + u0 * ldcb, bytes, &bar[0]);
    issued[0] = 1;
    if (cnt > 1) {
      bulk::load(slices + ldcb, cb + (u0 + G) * ldcb, bytes, &bar[1]);
      issued[1] = 1;
    }
  }
  bool fail = false;
  if (half == 1) {  // the wait's outcome is made warp-uniform before the shuffles
    if (__all_sync(0xffffffffu, tc::mbar_wait(&bar[0], 0, kCopyWaitLimit))) column_inverse<N, XM>(slices, jidx, l, live, h, tiles, tw);
    else fail = true;
  }
  bool stop = __syncthreads_or(fail);
  for (int k = 0; k < cnt && !stop; ++k) {
    const long u = u0 + (long)k * G;
    const int z = (int)(u % g.n3);
    float2 *tcur = tiles + (k & 1) * N * NX;
    row_vloc<N, XM>(tcur, t >> 1, h, pa.field + ((size_t)z * N + (size_t)(t >> 1)) * N, tw);
    __syncthreads();
    float2 *scur = slices + (k % 3) * ldcb;
    if (half == 0) {
      column_forward<N, XM>(scur, jidx, l, live, h, tcur, tw);
      tc::fence_proxy_async();
    } else if (k + 1 < cnt) {
      const int b = (k + 1) % 3;
      if (__all_sync(0xffffffffu, tc::mbar_wait(&bar[b], (uint32_t)(((k + 1) / 3) & 1), kCopyWaitLimit)))
        column_inverse<N, XM>(slices + b * ldcb, jidx, l, live, h, tiles + ((k + 1) & 1) * N * NX, tw);
      else
        fail = true;
    }
    stop = __syncthreads_or(fail);
    if (stop) break;
    if (t == 0) {
      bulk::store(cb + u * ldcb, scur, bytes);
      if (k + 2 < cnt) {
        const int b = (k + 2) % 3;
        bulk::wait_read_but_one();  // the store of unit k - 1 from this slice has read it
        bulk::load(slices + b * ldcb, cb + (u + 2 * G) * ldcb, bytes, &bar[b]);
        ++issued[b];
      }
    }
  }
  if (t == 0) {
    if (stop) {  // let every load this block issued land before the block's shared memory goes away
#pragma unroll
      for (int b = 0; b < 3; ++b)
        if (issued[b] > 0) (void)tc::mbar_wait(&bar[b], (uint32_t)((issued[b] - 1) & 1), kCopyWaitLimit);
      atomicExch(err, 1);
    }
    bulk::wait_all();
  }
}

template <int N, int XM> size_t pipe2_smem(const Geo &g) {
  return sizeof(float2) * (3 * (size_t)g.ldcb + 2 * (size_t)N * (2 * XM + 1) + N) + 3 * sizeof(uint64_t);
}

template <int N, int XM> void pipe2_launch(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    WDF_CUDA_TRY(cudaGetDevice(&dev));
    WDF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t sm = pipe2_smem<N, XM>(f.g);
  int per_sm = 0;
  WDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plane_pipe2<N, XM>, 2 * N, sm));
  if (per_sm < 1) per_sm = 1;
  const long nunits = (long)npair * f.g.n3;
  const long grid = std::min<long>(nunits, (long)nsm * per_sm);
  launch_units("plane_vloc", 32, nunits, k_plane_pipe2<N, XM>, dim3((unsigned)grid), dim3(2 * N), sm, st, f.g, f.tw1, f.jidx, pa,
               nunits, f.err);
  WDF_CUDA_TRY(cudaGetLastError());
}

bool pipe2_enabled() {
  static const bool on = std::getenv("WDF_NO_PIPE_PLANE") == nullptr;
  return on;
}

}  // namespace

// the (N, disk bound) pairs this kernel is compiled for
#define WDF_PIPE2_SIZES(X) X(96, 22)

bool plane_pipe2_available(const Geo &g, const int *err) {
  if (!pipe2_enabled() || err == nullptr || g.n1 != g.n2) return false;
  if (g.ymax > g.xmax || g.nxact != 2 * g.xmax + 1 || g.ldcb % 2 != 0) return false;
#define X(N, XM) \
  if (g.n1 == N && g.xmax == XM) return true;
  WDF_PIPE2_SIZES(X)
#undef X
  return false;
}

void set_plane_pipe2_limits(const Geo &g) {
#define X(N, XM) \
  if (g.n1 == N && g.n2 == N) raise_smem_limit(k_plane_pipe2<N, XM>, pipe2_smem<N, XM>(g));
  WDF_PIPE2_SIZES(X)
#undef X
}

bool launch_plane_pipe2(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st) {
  if (npair <= 0 || !plane_pipe2_available(f.g, f.err)) return false;
#define X(N, XM)                       \
  if (f.g.n1 == N && f.g.xmax == XM) { \
    pipe2_launch<N, XM>(f, npair, pa, st); \
    return true;                       \
  }
  WDF_PIPE2_SIZES(X)
#undef X
  return false;
}

}  // namespace wdf

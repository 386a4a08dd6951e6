// Persistent FP32 V_loc plane kernel for 64 x 64 planes whose occupied columns are the full disk
// |n1|, |n2| <= XM (cubic and other cells whose sphere projection is a full disk; XM <= 15).
//
// The work is the same as k_plane_reg's: for one z plane of one Gamma pair, the inverse n2
// transform of the occupied x columns, the inverse n1 transform of every row, the product with
// V_loc(r), the forward n1 transform and the forward n2 transform of the occupied columns back to
// the column buffer. This kernel reorganises it in three ways:
//  * Persistent blocks with a static round-robin over the (pair, plane) units; each unit's slice of
//    the column buffer (ldcb contiguous complex values) moves into and out of shared memory with
//    bulk asynchronous copies (cp.async.bulk, completion on an mbarrier for loads and bulk groups
//    for stores), three slices in flight, so the column gathers and scatters are shared-memory
//    accesses and the global latency hides behind the transforms of the previous unit.
//  * The column phases of consecutive units overlap: warp 0 runs the forward n2 transforms of
//    unit k while warp 1 runs the inverse n2 transforms of unit k + 1, two tiles in shared memory;
//    per unit the block spends one column-transform time instead of two.
//  * The tile keeps only the 2 XM + 1 occupied columns (odd pitch: conflict-free column and row
//    access), and the disk bound is a compile-time constant, so the zero inputs of the inverse
//    transforms and the unused outputs of the forward transforms drop out of the arithmetic.
// Every wait is bounded: a block whose copy does not complete sets the error flag, waits (again
// bounded) for the copies it has in flight and leaves.
#include <cstdlib>

#include "fft.cuh"
#include "kernels.cuh"
#include "plane_reg.cuh"
#include "tc.cuh"

namespace wdf {
namespace {

using namespace tc;

constexpr int kN = 64;
constexpr long kCopyWaitLimit = 1L << 24;

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// all but the newest bulk store have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_but_one() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int XM> __device__ __forceinline__ constexpr bool on_disk(int i) { return i <= XM || i >= kN - XM; }
// compact column of natural index x on the disk
template <int XM> __device__ __forceinline__ constexpr int compact(int x) { return x <= XM ? x : x - (kN - (2 * XM + 1)); }

// inverse n2 transform of compact column l (natural x): slice -> tile column l, rows in natural order
template <int XM>
__device__ __forceinline__ void column_inverse(const float2 *sl, const int *__restrict__ jidx, int l, float2 *tile, const float2 *tw) {
  constexpr int NX = 2 * XM + 1;
  const int x = l <= XM ? l : l + (kN - NX);
  float2 v[kN];
#pragma unroll
  for (int y = 0; y < kN; ++y) {
    if (on_disk<XM>(y)) {
      const int jj = __ldg(jidx + y * kN + x);
      v[y] = jj >= 0 ? sl[jj] : make_float2(0.f, 0.f);
    } else {
      v[y] = make_float2(0.f, 0.f);
    }
  }
  line_inverse<kN>(v, tw);
#pragma unroll
  for (int s = 0; s < kN; ++s) tile[perm_index<kN>(s) * NX + l] = v[s];
}

// forward n2 transform of compact column l back into the slice
template <int XM>
__device__ __forceinline__ void column_forward(float2 *sl, const int *__restrict__ jidx, int l, const float2 *tile, const float2 *tw) {
  constexpr int NX = 2 * XM + 1;
  const int x = l <= XM ? l : l + (kN - NX);
  float2 v[kN];
#pragma unroll
  for (int s = 0; s < kN; ++s) v[s] = tile[perm_index<kN>(s) * NX + l];
  line_forward<kN>(v, tw);
#pragma unroll
  for (int y = 0; y < kN; ++y) {
    if (on_disk<XM>(y)) {
      const int jj = __ldg(jidx + y * kN + x);
      if (jj >= 0) sl[jj] = v[y];
    }
  }
}

// row y of the tile: inverse n1 transform, V_loc(r) product, forward n1 transform
template <int XM>
__device__ __forceinline__ void row_vloc(float2 *tile, int y, const float *__restrict__ vrow, const float2 *tw) {
  constexpr int NX = 2 * XM + 1;
  float2 *tr = tile + y * NX;
  float2 v[kN];
#pragma unroll
  for (int x = 0; x < kN; ++x) v[x] = on_disk<XM>(x) ? tr[compact<XM>(x)] : make_float2(0.f, 0.f);
  line_inverse<kN>(v, tw);
  const float4 *v4 = reinterpret_cast<const float4 *>(vrow);
#pragma unroll
  for (int c = 0; c < kN / 4; ++c) {
    const float4 w = __ldg(v4 + c);
    const float we[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int x = 4 * c + e, s = 8 * (x % 8) + x / 8;  // slot holding natural x after line_inverse
      v[s] = cscal<float>(v[s], we[e]);
    }
  }
  line_forward<kN>(v, tw);
#pragma unroll
  for (int x = 0; x < kN; ++x)
    if (on_disk<XM>(x)) tr[compact<XM>(x)] = v[x];
}

template <int XM>
__global__ void __launch_bounds__(kN, 4) k_plane_pipe(Geo g, const float2 *__restrict__ twg, const int *__restrict__ jidx,
                                                      PlaneArgs<float> pa, long nunits, int *err) {
  constexpr int NX = 2 * XM + 1;
  static_assert(NX <= 32, "one warp per column phase");
  extern __shared__ __align__(128) unsigned char smraw[];
  const int ldcb = g.ldcb;
  float2 *slices = reinterpret_cast<float2 *>(smraw);  // 3 x ldcb
  float2 *tiles = slices + 3 * ldcb;                     // 2 x kN x NX
  float2 *tw = tiles + 2 * kN * NX;                      // kN
  uint64_t *bar = reinterpret_cast<uint64_t *>(tw + kN);  // 3
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long G = gridDim.x, u0 = blockIdx.x;
  if (u0 >= nunits) return;
  const int cnt = (int)((nunits - 1 - u0) / G) + 1;
  const uint32_t bytes = (uint32_t)ldcb * (uint32_t)sizeof(float2);
  float2 *cb = pa.cb;
  int issued[3] = {0, 0, 0};  // loads issued into each slice (thread 0)
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  tw[t] = twg[t];
  __syncthreads();
  if (t == 0) {
    bulk_load(slices, cb + u0 * ldcb, bytes, &bar[0]);
    issued[0] = 1;
    if (cnt > 1) {
      bulk_load(slices + ldcb, cb + (u0 + G) * ldcb, bytes, &bar[1]);
      issued[1] = 1;
    }
  }
  bool fail = false;
  if (warp == 1 && lane < NX) {
    if (mbar_wait(&bar[0], 0, kCopyWaitLimit)) column_inverse<XM>(slices, jidx, lane, tiles, tw);
    else fail = true;
  }
  bool stop = __syncthreads_or(fail);
  for (int k = 0; k < cnt && !stop; ++k) {
    const long u = u0 + (long)k * G;
    const int z = (int)(u % g.n3);
    float2 *tcur = tiles + (k & 1) * kN * NX;
    row_vloc<XM>(tcur, t, pa.field + (size_t)z * kN * kN + (size_t)t * kN, tw);
    __syncthreads();
    float2 *scur = slices + (k % 3) * ldcb;
    if (warp == 0) {
      if (lane < NX) column_forward<XM>(scur, jidx, lane, tcur, tw);
      fence_proxy_async();
    } else if (k + 1 < cnt && lane < NX) {
      const int b = (k + 1) % 3;
      if (mbar_wait(&bar[b], (uint32_t)(((k + 1) / 3) & 1), kCopyWaitLimit))
        column_inverse<XM>(slices + b * ldcb, jidx, lane, tiles + ((k + 1) & 1) * kN * NX, tw);
      else
        fail = true;
    }
    stop = __syncthreads_or(fail);
    if (stop) break;
    if (t == 0) {
      bulk_store(cb + u * ldcb, scur, bytes);
      if (k + 2 < cnt) {
        const int b = (k + 2) % 3;
        bulk_wait_read_but_one();  // the store of unit k - 1 from this slice has read it
        bulk_load(slices + b * ldcb, cb + (u + 2 * G) * ldcb, bytes, &bar[b]);
        ++issued[b];
      }
    }
  }
  if (t == 0) {
    if (stop) {  // let every load this block issued land before the block's shared memory goes away
      bool ok = true;
#pragma unroll
      for (int b = 0; b < 3; ++b)
        if (issued[b] > 0) ok &= mbar_wait(&bar[b], (uint32_t)((issued[b] - 1) & 1), kCopyWaitLimit);
      (void)ok;
      atomicExch(err, 1);
    }
    bulk_wait_all();
  }
}

template <int XM> size_t pipe_smem(const Geo &g) {
  return sizeof(float2) * (3 * (size_t)g.ldcb + 2 * (size_t)kN * (2 * XM + 1) + kN) + 3 * sizeof(uint64_t);
}

template <int XM> void pipe_launch(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    WDF_CUDA_TRY(cudaGetDevice(&dev));
    WDF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t sm = pipe_smem<XM>(f.g);
  int per_sm = 0;
  WDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plane_pipe<XM>, kN, sm));
  if (per_sm < 1) per_sm = 1;
  const long nunits = (long)npair * f.g.n3;
  const long grid = std::min<long>(nunits, (long)nsm * per_sm);
  launch_units("plane_vloc", 32, nunits, k_plane_pipe<XM>, dim3((unsigned)grid), dim3(kN), sm, st, f.g, f.tw1, f.jidx, pa, nunits,
               f.err);
  WDF_CUDA_TRY(cudaGetLastError());
}

bool pipe_enabled() {
  static const bool on = std::getenv("WDF_NO_PIPE_PLANE") == nullptr;
  return on;
}

}  // namespace

// the disk bounds this kernel is compiled for (64 x 64 planes)
#define WDF_PIPE_XM(X) X(14) X(15)

bool plane_pipe_available(const Geo &g, const int *err) {
  if (!pipe_enabled() || err == nullptr || g.n1 != kN || g.n2 != kN) return false;
  if (g.ymax > g.xmax || g.nxact != 2 * g.xmax + 1 || g.ldcb % 2 != 0) return false;
  switch (g.xmax) {
#define X(XM) case XM:
    WDF_PIPE_XM(X)
#undef X
    return true;
    default: return false;
  }
}

void set_plane_pipe_limits(const Geo &g) {
  if (g.n1 != kN || g.n2 != kN) return;
#define X(XM) raise_smem_limit(k_plane_pipe<XM>, pipe_smem<XM>(g));
  WDF_PIPE_XM(X)
#undef X
}

bool launch_plane_pipe(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st) {
  if (npair <= 0 || !plane_pipe_available(f.g, f.err)) return false;
  switch (f.g.xmax) {
#define X(XM) \
  case XM: pipe_launch<XM>(f, npair, pa, st); return true;
    WDF_PIPE_XM(X)
#undef X
    default: return false;
  }
}

}  // namespace wdf

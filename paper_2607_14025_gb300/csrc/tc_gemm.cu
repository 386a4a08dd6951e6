// Tensor-core (tcgen05, kind::tf32) forms of the two dense products of the FP32 inner CG:
//   gram:    S[j][s] = sum_e w_e Re(conj(U_j[e]) X_s[e])       (projections on [beta; psi])
//   lincomb: Y_s = c0 Y_s + sum_j U_j S[j][s] d_j               (KB term and alpha P shift)
// Complex vectors are read as real rows of 2 N_int values, so both are real GEMMs with K-major
// operands. FP32 accuracy from TF32 units by the three-term split a b ~ a_h b_h + a_h b_l + a_l b_h
// with a_h the upper 19 bits of a and a_l = a - a_h (the dropped a_l b_l is ~2^-22 |a b|).
// Operand tiles arrive in 64-byte-swizzled shared memory by tensor-memory-access copies (tensor
// maps made per launch; reads past a matrix's end give zeros), four stages deep, in
// warp-specialised pipelines coupled by mbarriers: one thread loads, one thread issues the MMAs
// and commits them to the stage's mbarrier; accumulators sit in TMEM and the epilogues read them
// with tcgen05.ld. Every mbarrier wait is bounded: on expiry the kernel raises a flag, waits
// (bounded) for what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "engine.cuh"
#include "tc.cuh"

namespace wdf {

namespace {

constexpr int TM = 128;              // MMA M: solves per tile
constexpr long kWaitLimit = 1L << 26;  // polls of an mbarrier before giving up
// chunks (of 16 K values) per FP32 accumulation chain of the Gram: longer chains lose accuracy
// (the sums run over 2 N_int products), so every kPromote chunks (2,048 K values) the partial sums
// move into the FP64 output
constexpr int kPromote = 128;

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return (unsigned char *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// S (+ split partials) = U_w X^T; grid (solve tiles, splits, chunks of U rows). Warp-specialised
// pipeline over kGramStages shared-memory stages of kGramK values (64-byte swizzled K-major rows):
//   warp 0   one thread loads the X, U hi and U lo tiles of a stage with tensor-memory-access
//            copies (cp.async.bulk.tensor, completion counted in bytes on the stage's full barrier);
//   warp 1   one thread issues the stage's 3 x 2 MMAs (hi hi, hi lo, lo hi) and commits them to the
//            stage's empty barrier (the loader's go-ahead to refill it);
//   warps 4-7 make the low parts of X in shared memory once a stage has landed (lo barrier);
//   warps 8-11 move each finished FP32 accumulation chain (kPromote stages) from its TMEM half into
//            the FP64 output (the first chain stores, later ones add) while the MMAs fill the
//            other half, then release the half (tfree barrier).
// No thread waits on another through a block-wide barrier inside the loop; every mbarrier wait is
// bounded and a role that gives up makes the others give up at their next wait.
constexpr int kGramK = 16;                 // K values per stage (one 64-byte row)
constexpr int kGramStages = 4;
constexpr int kGramXB = TM * kGramK * 4;   // bytes of the 128-row X stage
constexpr int kGramThreads = 384;

// blockIdx.z picks a chunk of rows of U (rows z nbox ...; nbox <= kGramRows, the chunks as even as
// multiples of 32 allow): a CTA holds the accumulators of 128 solves x one chunk in TMEM, so U of
// any height runs in chunks.
constexpr int kGramRows = 256;

__host__ __device__ constexpr int gram_stage_bytes(int nbox) { return 2 * kGramXB + 2 * nbox * kGramK * 4; }

__device__ __forceinline__ void tma_load2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(map), "r"(x), "r"(y), "r"(tc::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// nbox: rows of the U boxes the tensor maps load (the stage layout); na_all: rows of U
__global__ void __launch_bounds__(kGramThreads, 1) k_gram_tc(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mUh,
                                                             const __grid_constant__ CUtensorMap mUl, Geo g, int nb, int na_all, int nbox,
                                                             double *__restrict__ out, int ldo, int ch_per_split, size_t split_stride,
                                                             int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = align1024(smraw);
  const int j0 = blockIdx.z * nbox;
  const int na = min(nbox, na_all - j0), nu = ((na + 31) / 32) * 32;
  out += (size_t)j0 * ldo;
  const int UB = nbox * kGramK * 4, SB = gram_stage_bytes(nbox);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + kGramStages * SB);
  uint64_t *lo = full + kGramStages, *empty = lo + kGramStages, *chain = empty + kGramStages, *tfree = chain + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(tfree + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * TM;
  const int kf = 2 * g.nint;
  const int nch = (kf + kGramK - 1) / kGramK;
  const int c0 = blockIdx.y * ch_per_split, c1 = min(nch, c0 + ch_per_split);
  const int n = max(0, c1 - c0);
  const int nchains = (n + kPromote - 1) / kPromote;
  if (tid == 0) {
    for (int i = 0; i < kGramStages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&lo[i], 4);
      tc::mbar_init(&empty[i], 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&chain[h], 1);
      tc::mbar_init(&tfree[h], 4);
    }
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  bool fail = false;
  if (warp == 0) {
    if (lane == 0) {  // loads
      int issued = 0;
      for (int i = 0; i < n; ++i) {
        const int st = i % kGramStages, k = i / kGramStages;
        if (k > 0 && !tc::mbar_wait(&empty[st], (k - 1) & 1, kWaitLimit)) {
          fail = true;
          break;
        }
        unsigned char *S = sm + st * SB;
        const int f0 = (c0 + i) * kGramK;
        mbar_expect_tx(&full[st], (uint32_t)(kGramXB + 2 * UB));
        tma_load2d(S, &mX, f0, s0, &full[st]);
        tma_load2d(S + 2 * kGramXB, &mUh, f0, j0, &full[st]);
        tma_load2d(S + 2 * kGramXB + UB, &mUl, f0, j0, &full[st]);
        issued = i + 1;
      }
      // every copy issued lands before the block's shared memory goes away
      for (int i = max(0, issued - kGramStages); i < issued; ++i)
        if (!tc::mbar_wait(&full[i % kGramStages], (i / kGramStages) & 1, kWaitLimit)) fail = true;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMAs
      const uint32_t idesc = tc::idesc_tf32(TM, nu);
      int issued = 0;
      for (int i = 0; i < n; ++i) {
        const int st = i % kGramStages, k = i / kGramStages, p = i / kPromote, first = i % kPromote;
        if (first == 0 && p >= 2 && !tc::mbar_wait(&tfree[p & 1], ((p - 2) >> 1) & 1, kWaitLimit)) {
          fail = true;
          break;
        }
        if (!tc::mbar_wait(&lo[st], k & 1, kWaitLimit)) {
          fail = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t base = tc::smem_u32(sm + st * SB);
        const uint32_t acc = tmem + (uint32_t)((p & 1) * 256);
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t a = base + (term == 2 ? kGramXB : 0), b = base + 2 * kGramXB + (term == 1 ? UB : 0);
#pragma unroll
          for (int ks = 0; ks < kGramK / 8; ++ks)
            tc::mma_tf32(acc, tc::desc_sw64(a + 32 * ks), tc::desc_sw64(b + 32 * ks), idesc, (first | term | ks) ? 1u : 0u);
        }
        tc::mma_commit(&empty[st]);
        if (first == kPromote - 1 || i == n - 1) tc::mma_commit(&chain[p & 1]);
        issued = i + 1;
      }
      if (issued > 0 && !tc::mbar_wait(&empty[(issued - 1) % kGramStages], ((issued - 1) / kGramStages) & 1, kWaitLimit))
        fail = true;  // the MMAs issued have finished with TMEM and shared memory
    }
  } else if (warp >= 4 && warp < 8) {  // low parts of X
    const int t0 = tid - 128;
    for (int i = 0; i < n; ++i) {
      const int st = i % kGramStages, k = i / kGramStages;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[st], k & 1, kWaitLimit))) {
        fail = true;
        break;
      }
      unsigned char *S = sm + st * SB;
#pragma unroll
      for (int u = 0; u < kGramXB / 16 / 128; ++u) {
        const int t = t0 + 128 * u;
        const float4 v = *reinterpret_cast<const float4 *>(S + 16 * t);
        *reinterpret_cast<float4 *>(S + kGramXB + 16 * t) =
            make_float4(tc::tf32_low(v.x), tc::tf32_low(v.y), tc::tf32_low(v.z), tc::tf32_low(v.w));
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&lo[st]);
    }
  } else if (warp >= 8) {  // finished chains out of TMEM; warp w reads TMEM lanes 32 (w mod 4) ...
    const int qd = warp & 3, orow = 32 * qd + lane, osol = s0 + orow;
    double *o = out + (size_t)blockIdx.y * split_stride;
    for (int p = 0; p < nchains; ++p) {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&chain[p & 1], (p >> 1) & 1, kWaitLimit))) {
        fail = true;
        break;
      }
      tc::fence_after_sync();
      const uint32_t base = tmem + (uint32_t)((p & 1) * 256) + ((uint32_t)(32 * qd) << 16);
      for (int col = 0; col < nu; col += 16) {
        float v[16];
        tc::tmem_ld16(base + (uint32_t)col, v);
        if (osol < nb) {
          double old[16];  // all loads in flight before the adds and stores
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) old[kk] = (p > 0 && col + kk < na) ? o[(size_t)(col + kk) * ldo + osol] : 0.0;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk)
            if (col + kk < na) o[(size_t)(col + kk) * ldo + osol] = old[kk] + (double)v[kk];
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[p & 1]);
    }
    if (n == 0 && osol < nb)  // an empty K range still owns its part of the output
      for (int col = 0; col < na; ++col) o[(size_t)col * ldo + osol] = 0.0;
  }
  fail = __syncthreads_or(fail);
  if (fail && tid == 0) atomicExch(err, 1);
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

__global__ void k_tc_sum_splits(const double *__restrict__ work, int nsplit, size_t stride, double *__restrict__ out, int na, int nb,
                                int ldo) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)na * nb) return;
  const int j = (int)(t / nb), s = (int)(t % nb);
  double a = 0.0;
  for (int k = 0; k < nsplit; ++k) a += work[k * stride + (size_t)j * ldo + s];
  out[(size_t)j * ldo + s] = a;
}

// Cd[s][j] = S[j][s] d_j (j < na, else 0), hi and lo parts, through a 32 x 32 shared tile
__global__ void k_tc_coef(const double *__restrict__ S, int ldc, const double *__restrict__ d, int na, int nb, int kp,
                          float *__restrict__ hi, float *__restrict__ lo) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.y * 32, s0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, s = s0 + threadIdx.x;
    float v = 0.f;
    if (j < na && s < nb) v = (float)(S[(size_t)j * ldc + s] * (d ? d[j] : 1.0));
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int s = s0 + r, j = j0 + threadIdx.x;
    if (s < nb && j < kp) {
      const float v = tile[threadIdx.x][r];
      hi[(size_t)s * kp + j] = v;
      lo[(size_t)s * kp + j] = tc::tf32_low(v);
    }
  }
}

// Y = c0 Y + Cd Ut^T on float rows (2 N_int), partial <P_s, Y_s> per 128-element tile;
// grid (solve tiles, 256-value tiles), 256 threads. The K loop (K = rows of U, in stages of
// kGramK values, kGramStages deep) is warp-specialised: one thread of warp 0 loads the C (hi, lo)
// and U^T (hi, lo) tiles with tensor-memory-access copies, one thread of warp 1 issues the MMAs;
// the finished tile goes TMEM -> shared memory, then each warp updates whole rows of Y with
// coalesced accesses and reduces its row's partial inner product.
constexpr int DP = 260;  // shared row pitch of the result tile (floats): conflict-free float4 stores
constexpr int kLinTN = 256;
constexpr int kLinAB = TM * kGramK * 4, kLinBB = kLinTN * kGramK * 4, kLinSB = 2 * kLinAB + 2 * kLinBB;

__global__ void __launch_bounds__(256, 1) k_lincomb_tc(const __grid_constant__ CUtensorMap mCh, const __grid_constant__ CUtensorMap mCl,
                                                       const __grid_constant__ CUtensorMap mUh, const __grid_constant__ CUtensorMap mUl,
                                                       Geo g, float *__restrict__ Y, int ny, int kp, float c0, const float *__restrict__ P,
                                                       double *__restrict__ part, int nchunk, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = align1024(smraw);
  constexpr int TN = kLinTN;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + kGramStages * kLinSB);
  uint64_t *empty = full + kGramStages, *done_bar = empty + kGramStages;
  uint32_t *slot = reinterpret_cast<uint32_t *>(done_bar + 1);
  float *D = reinterpret_cast<float *>(sm);  // result tile [128][DP], over the operand stages
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * TM, f0 = blockIdx.y * TN;
  const int kf = 2 * g.nint, ldf = 2 * g.ld;
  const int nkc = kp / kGramK;
  if (tid == 0) {
    for (int i = 0; i < kGramStages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done_bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(slot, 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  bool fail = false;
  if (warp == 0 && lane == 0) {  // loads
    int issued = 0;
    for (int i = 0; i < nkc; ++i) {
      const int st = i % kGramStages, k = i / kGramStages;
      if (k > 0 && !tc::mbar_wait(&empty[st], (k - 1) & 1, kWaitLimit)) {
        fail = true;
        break;
      }
      unsigned char *S = sm + st * kLinSB;
      const int k0 = i * kGramK;
      mbar_expect_tx(&full[st], (uint32_t)kLinSB);
      tma_load2d(S, &mCh, k0, s0, &full[st]);
      tma_load2d(S + kLinAB, &mCl, k0, s0, &full[st]);
      tma_load2d(S + 2 * kLinAB, &mUh, k0, f0, &full[st]);
      tma_load2d(S + 2 * kLinAB + kLinBB, &mUl, k0, f0, &full[st]);
      issued = i + 1;
    }
    for (int i = max(0, issued - kGramStages); i < issued; ++i)
      if (!tc::mbar_wait(&full[i % kGramStages], (i / kGramStages) & 1, kWaitLimit)) fail = true;
  } else if (warp == 1 && lane == 0) {  // MMAs: hi hi, hi lo, lo hi
    const uint32_t idesc = tc::idesc_tf32(TM, TN);
    int issued = 0;
    for (int i = 0; i < nkc; ++i) {
      const int st = i % kGramStages, k = i / kGramStages;
      if (!tc::mbar_wait(&full[st], k & 1, kWaitLimit)) {
        fail = true;
        break;
      }
      tc::fence_after_sync();
      const uint32_t base = tc::smem_u32(sm + st * kLinSB);
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const uint32_t a = base + (term == 2 ? kLinAB : 0), b = base + 2 * kLinAB + (term == 1 ? kLinBB : 0);
#pragma unroll
        for (int ks = 0; ks < kGramK / 8; ++ks)
          tc::mma_tf32(tmem, tc::desc_sw64(a + 32 * ks), tc::desc_sw64(b + 32 * ks), idesc, (i | term | ks) ? 1u : 0u);
      }
      tc::mma_commit(&empty[st]);
      issued = i + 1;
    }
    if (issued == nkc) tc::mma_commit(done_bar);  // arrives once every MMA has completed
    else if (issued > 0)
      (void)tc::mbar_wait(&empty[(issued - 1) % kGramStages], ((issued - 1) / kGramStages) & 1, kWaitLimit);
  }
  fail = __syncthreads_or(fail);
  bool done = !fail && (nkc == 0 || tc::mbar_wait(done_bar, 0, kWaitLimit));
  done = __syncthreads_and(done);
  if (done) {
    // every MMA has completed, so the operand stages are free: TMEM -> D[128][DP]
    tc::fence_after_sync();
    const int qd = warp & 3, h = warp >> 2, row = 32 * qd + lane;
    for (int cg = 0; cg < TN / 2; cg += 16) {
      const int col = h * (TN / 2) + cg;
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)col, v);
#pragma unroll
      for (int k = 0; k < 16; k += 4) *reinterpret_cast<float4 *>(D + row * DP + col + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  __syncthreads();
  if (done) {
    // warp w updates rows w, w + 8, ...: lane l owns values 8 l .. 8 l + 7 of the 256. Four rows
    // at a time: every global load of the four (old Y, P) is issued before their arithmetic and
    // stores, so they are in flight together
    constexpr int RB = 4;
    for (int r0 = warp; r0 < TM; r0 += 8 * RB) {
      float4 yo[RB][2], pv[RB][2];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int s = s0 + r0 + 8 * u;
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
          const int f = 8 * lane + 4 * hq;  // 4 values = 2 complex elements
          yo[u][hq] = pv[u][hq] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (s < ny && f0 + f < kf) {  // a tail piece reads one element of row padding (kf is even)
            if (c0 != 0.f) yo[u][hq] = *reinterpret_cast<const float4 *>(Y + (size_t)s * ldf + f0 + f);
            if (P) pv[u][hq] = *reinterpret_cast<const float4 *>(P + (size_t)s * ldf + f0 + f);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int r = r0 + 8 * u, s = s0 + r;
        if (s >= ny) break;  // rows are in order: the rest of this warp's rows are past the end too
        float *y = Y + (size_t)s * ldf + f0;
        float dsum = 0.f;  // a lane adds at most 4 products; the warp sum is FP64
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
          const int f = 8 * lane + 4 * hq;
          if (f0 + f < kf) {
            float4 d = *reinterpret_cast<const float4 *>(D + r * DP + f);
            if (f0 + f + 3 >= kf) d.z = d.w = 0.f;  // one element past the end
            float4 yv = d;
            if (c0 != 0.f) {
              const float4 o = yo[u][hq];
              yv = make_float4(fmaf(c0, o.x, d.x), fmaf(c0, o.y, d.y), fmaf(c0, o.z, d.z), fmaf(c0, o.w, d.w));
            }
            if (f0 + f + 3 < kf) {
              *reinterpret_cast<float4 *>(y + f) = yv;
            } else {
              *reinterpret_cast<float2 *>(y + f) = make_float2(yv.x, yv.y);
            }
            if (P) {
              const int e = (f0 + f) >> 1;
              const float4 q4 = pv[u][hq];
              const float w0 = e < g.len0 ? 1.f : 2.f, w1 = e + 1 < g.len0 ? 1.f : 2.f;
              dsum += w0 * (q4.x * yv.x + q4.y * yv.y);
              if (f0 + f + 3 < kf) dsum += w1 * (q4.z * yv.z + q4.w * yv.w);
            }
          }
        }
        if (part) {
          double dd = (double)dsum;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
          if (lane == 0) part[(size_t)s * nchunk + blockIdx.y] = dd;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// U_w = w U (hi, lo) as [na][2 ld] and U^T (hi, lo) as [2 ld][kp], zero padded
__global__ void k_tc_prep_u(Geo g, const float2 *__restrict__ U, int na, int kp, float *__restrict__ uwh, float *__restrict__ uwl,
                            float *__restrict__ uth, float *__restrict__ utl) {
  const int ldf = 2 * g.ld;
  const size_t tot = (size_t)ldf * kp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / ldf), f = (int)(t % ldf), e = f >> 1;
    float v = 0.f;
    if (j < na && e < g.nint) {
      const float2 u = U[(size_t)j * g.ld + e];
      v = (f & 1) ? u.y : u.x;
    }
    if (j < na) {
      const float w = e < g.len0 ? v : 2.f * v;
      uwh[(size_t)j * ldf + f] = w;
      uwl[(size_t)j * ldf + f] = tc::tf32_low(w);
    }
    uth[(size_t)f * kp + j] = v;
    utl[(size_t)f * kp + j] = tc::tf32_low(v);
  }
}

size_t gram_tc_smem(int nbox) { return 1024 + (size_t)kGramStages * gram_stage_bytes(nbox) + 8 * (3 * kGramStages + 4) + 16; }
size_t lincomb_tc_smem() {
  const size_t stages = (size_t)kGramStages * kLinSB, tile = sizeof(float) * (size_t)TM * DP;
  return 1024 + std::max(stages, tile) + 8 * (2 * kGramStages + 1) + 16;
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

bool tc_enabled() {
  static const bool on = std::getenv("WDF_NO_TC") == nullptr;
  return on && tmap_encoder() != nullptr;
}

int tc_rows(int na) { return ((na + 31) / 32) * 32; }

void set_tc_limits() {
  raise_smem_limit(k_gram_tc, (size_t)((int)gram_tc_smem(256)));
  raise_smem_limit(k_lincomb_tc, (size_t)((int)lincomb_tc_smem()));
}

void launch_tc_prep_u(const Geo &g, const float2 *U, int na, float *uwh, float *uwl, float *uth, float *utl, cudaStream_t st) {
  const int kp = tc_rows(na);
  launch("tc_prep", 32, k_tc_prep_u, dim3(2048), dim3(256), 0, st, g, U, na, kp, uwh, uwl, uth, utl);
  WDF_CUDA_TRY(cudaGetLastError());
}

// K splits of the Gram: one CTA per SM (shared memory), so the launch runs in waves of nsm CTAs;
// choose the split count (at most nch / 16, so that each CTA keeps a pipeline of >= 16 chunks)
// that minimises waves x (chunks per CTA + 12), the 12 standing for a CTA's partial-sum write
// (128 x 192 doubles, about the bytes of two dozen 16-value X chunks, written without waiting),
// the smaller count on ties (fewer partial sums to add)
static int gram_tc_splits(int nch, int tiles) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  const int smax = std::max(1, std::min(nch / 16, 4 * ((nsm + tiles - 1) / tiles)));
  long best = -1;
  int bs = 1;
  for (int sp = 1; sp <= smax; ++sp) {
    const long waves = ((long)tiles * sp + nsm - 1) / nsm, per = (nch + sp - 1) / sp;
    const long cost = waves * (per + 12);
    if (best < 0 || cost < best) {
      best = cost;
      bs = sp;
    }
  }
  return bs;
}

size_t gram_tc_work_doubles(const Geo &g, int na, int nb) {
  const int nch = (2 * g.nint + kGramK - 1) / kGramK;
  const int tiles = ((nb + TM - 1) / TM) * ((na + kGramRows - 1) / kGramRows);
  const int nsplit = gram_tc_splits(nch, tiles);
  return nsplit > 1 ? (size_t)nsplit * na * nb : 0;
}

// rows of kf FP32 values with ldf values between row starts, read in boxes of kGramK x box_rows
// into 64-byte swizzled shared memory; reads past the last row or value return zeros
static CUtensorMap rows_map(const float *base, int kf, int rows, int ldf, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dim[2] = {(cuuint64_t)kf, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)ldf * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kGramK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = tmap_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dim, stride, box, es,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw ApiFailure(WDF_EINVAL, "tensor map encoding failed (" + std::to_string((int)r) + ")");
  return m;
}

void launch_gram_tc(const Geo &g, const float *X, int nb, const float *uwh, const float *uwl, int na, double *out, double *work,
                    size_t work_cap, int *err, cudaStream_t st) {
  if (nb <= 0 || na <= 0) return;
  const int nmc = (na + kGramRows - 1) / kGramRows;
  const int nbox = tc_rows((na + nmc - 1) / nmc);  // even chunks of U rows
  const int kf = 2 * g.nint, ldf = 2 * g.ld;
  const int nch = (kf + kGramK - 1) / kGramK;
  const int tiles = (nb + TM - 1) / TM;
  int nsplit = gram_tc_splits(nch, tiles * nmc);
  if ((size_t)nsplit * na * nb > work_cap) nsplit = 1;
  const int per = (nch + nsplit - 1) / nsplit;
  nsplit = (nch + per - 1) / per;
  const CUtensorMap mX = rows_map(X, kf, nb, ldf, TM), mUh = rows_map(uwh, kf, na, ldf, nbox), mUl = rows_map(uwl, kf, na, ldf, nbox);
  double *dst = nsplit == 1 ? out : work;
  const size_t stride = nsplit == 1 ? (size_t)0 : (size_t)na * nb;
  launch("gram", 32, k_gram_tc, dim3(tiles, nsplit, nmc), dim3(kGramThreads), gram_tc_smem(nbox), st, mX, mUh, mUl, g, nb, na, nbox, dst,
         nb, per, stride, err);
  WDF_CUDA_TRY(cudaGetLastError());
  if (nsplit > 1) {
    launch("gram_sum", 0, k_tc_sum_splits, dim3((unsigned)(((size_t)na * nb + 255) / 256)), dim3(256), 0, st, (const double *)work,
           nsplit, stride, out, na, nb, nb);
    WDF_CUDA_TRY(cudaGetLastError());
  }
}

void launch_lincomb_tc(const Geo &g, float *Y, int ny, const double *S, int ldc, const double *d, int na, float *chi, float *clo,
                       const float *uth, const float *utl, float c0, const float *P, double *part, int *err, cudaStream_t st) {
  if (ny <= 0) return;
  const int kp = tc_rows(na);
  launch("lincomb", 32, k_tc_coef, dim3((ny + 31) / 32, (kp + 31) / 32), dim3(32, 8), 0, st, S, ldc, d, na, ny, kp, chi, clo);
  WDF_CUDA_TRY(cudaGetLastError());
  const int ntile = (2 * g.nint + kLinTN - 1) / kLinTN;
  const CUtensorMap mCh = rows_map(chi, kp, ny, kp, TM), mCl = rows_map(clo, kp, ny, kp, TM);
  const CUtensorMap mUh = rows_map(uth, kp, 2 * g.ld, kp, kLinTN), mUl = rows_map(utl, kp, 2 * g.ld, kp, kLinTN);
  launch("lincomb", 32, k_lincomb_tc, dim3((ny + TM - 1) / TM, ntile), dim3(256), lincomb_tc_smem(), st, mCh, mCl, mUh, mUl, g, Y, ny, kp,
         c0, P, part, lincomb_dot_chunks(g), err);
  WDF_CUDA_TRY(cudaGetLastError());
}

}  // namespace wdf

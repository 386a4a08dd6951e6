// Double-float projections of the residual and right-hand-side stages on the tensor cores, by
// exact integer slices (the error-free splitting of Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59, 2012, with the products summed exactly in the tensor cores' FP32 accumulators):
//   gram:    S[j][s] = sum_f uw[j][f] x[s][f]              (projections on [beta; psi], FP64 out)
//   lincomb: Y[s][f] = c0 Y[s][f] + sum_j C[s][j] u[j][f]  (C = S d; double-float Y)
// over the real rows of 2 N_int values of the complex vectors (the Gamma-point weights folded
// into uw), as on the CUDA cores, to the same ~2^-48 accuracy.
//
// Slices. A row r of a matrix with K values gets an exponent E_r (every |v| < 2^E_r) and T signed
// digits: v ~ sum_t m_t 2^(E_r - 7 (t + 1)), the integer round(v 2^(7T - E_r)) written in balanced
// base 128 (|m_0| <= 128, |m_t| <= 64 for t >= 1), so the fixed-point error is at most 2^(E_r - 7T).
// Every digit is an integer of at most 8 bits, exact in bf16. A product of two digits is an
// integer of at most 14 bits; products (t, u) of one "group" g = t + u carry the same power of
// two, 2^(E_a + E_b - 14 - 7 g). For g <= 3 a group's sum over a chain of 512 K values stays below
// 2^24 in magnitude (|m_0 m_0| <= 2^14; the g = 3 group has at most 6 x 2^12 per K value), so the
// tensor cores' FP32 accumulation of it is exact; after each chain the sums move into int32
// registers (exact while a split has at most 127 chains). Groups 4 .. T-1 are 2^-28 and less of
// group 0: they accumulate in FP32 with ordinary rounding. Products with t + u >= T are dropped
// (at most ~2^-47 of max|a| max|b| per term with T = 7).
//
// MMAs. For A digit t one tcgen05.mma (kind::f16, bf16 operands, FP32 accumulator, M = 128) runs
// against the B digits stacked in shared memory in descending order (block q holds digit
// T - 1 - q, 32 rows each), starting at block t: N = 32 (T - t) rows, whose accumulator column
// block b receives the product (t, T - 1 - t - b), i.e. group T - 1 - b for every t. So one
// accumulator block per group, T MMAs per 16 K values, T x 32 TMEM columns per chain; two chains
// alternate between the two halves of a 512-column allocation.
//
// Kernel roles (384 threads, one persistent CTA per SM walking the work items = tiles x K splits):
// warp 0 one thread loads the T A planes and the T B planes of a stage (32 K values) with
// tensor-memory-access copies; warp 1 one thread issues the MMAs; warps 4-11 move every finished
// chain out of TMEM (warp w: TMEM lanes 32 (w mod 4) .., columns 16 ((w - 4) / 4) .. of each
// 32-column block) and write each item's result after its last chain, while the MMAs of the next
// item fill the other TMEM half. Every mbarrier wait is bounded: on expiry the kernel raises the
// error flag, waits (bounded) for what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdlib>

#include "engine.cuh"
#include "tc.cuh"

namespace wdf {

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder();  // tc_gemm.cu

namespace {

constexpr int OZ_M = 128;       // A rows per tile (TMEM lanes)
constexpr int OZ_NB = 32;       // B rows per digit block
constexpr int OZ_KS = 32;       // K values per stage: one 64-byte row of bf16
constexpr int OZ_CHAIN = 16;    // stages per exact accumulation chain (512 K values)
constexpr int OZ_MAXCHAIN = 127;  // chains per split: the int32 sums stay exact
constexpr int OZ_THREADS = 384;
constexpr long kWaitLimit = 1L << 26;

template <int T> struct OzCfg {
  static constexpr int AB = OZ_M * OZ_KS * 2;   // bytes of one A digit plane of a stage
  static constexpr int BB = OZ_NB * OZ_KS * 2;  // bytes of one B digit block of a stage
  static constexpr int SB = T * (AB + BB);
  static constexpr int STAGES = T <= 7 ? 3 : 2;
  static_assert(T * OZ_NB <= 256, "accumulator blocks of one chain exceed half of TMEM");
};
template <int T> constexpr size_t oz_smem() { return 1024 + (size_t)OzCfg<T>::STAGES * OzCfg<T>::SB + 8 * (2 * OzCfg<T>::STAGES + 4) + 16; }

enum { OZ_GRAM = 0, OZ_LINCOMB = 1 };

struct OzArgs {
  int rowsA, rowsB;    // valid rows of A (M side) and B (N side)
  int tilesA, tilesB;  // tiles of 128 A rows and 32 B rows
  int groupA;          // A tiles per raster group (consecutive CTAs walk B within a group)
  int nst, per, nsplit;  // K stages in all, stages per split, splits
  const int *eA, *eB;  // row exponents
  double *out;         // gram: out[a][b] (split partials at + z split_stride)
  int ldo;
  size_t split_stride;
  df64 *Y;             // lincomb: Y[a][b] = c0 Y[a][b] + value
  size_t ldy;
  float c0;
  int *err;
};

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return (unsigned char *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}
__device__ __forceinline__ void tma_load3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          tc::smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
// instruction descriptor of kind::f16 with bf16 A and B, FP32 accumulator, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// an int32 as an exact double-float (the high part keeps the multiple of 256)
__device__ __forceinline__ df64 df_of_int(int v) {
  const int lo = v & 255;
  return df_two_sum((float)(v - lo), (float)lo);
}

// work item -> (A tile, B tile, K split): items enumerate tiles x splits; within a split a group
// of groupA A tiles walks every B tile (consecutive items share operands in L2)
struct OzItem {
  int a0, b0, z, c0, n;
};
__device__ __forceinline__ OzItem oz_item(const OzArgs &p, int item) {
  const int tiles = p.tilesA * p.tilesB;
  const int z = item / tiles, lin = item % tiles;
  const int gsz = p.groupA * p.tilesB, grp = lin / gsz, ingrp = lin % gsz;
  const int ga = min(p.groupA, p.tilesA - grp * p.groupA);
  OzItem it;
  it.a0 = (grp * p.groupA + ingrp % ga) * OZ_M;
  it.b0 = (ingrp / ga) * OZ_NB;
  it.z = z;
  it.c0 = z * p.per;
  it.n = max(0, min(p.nst, it.c0 + p.per) - it.c0);
  return it;
}

// persistent: CTA c takes items c, c + gridDim.x, ...; the stage ring and the chain counter run on
// across items, so the epilogue of one item overlaps the MMAs of the next
template <int T, int EPI>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                                                           OzArgs p) {
  typedef OzCfg<T> C;
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = align1024(smraw);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + C::STAGES * C::SB);
  uint64_t *empty = full + C::STAGES, *chain = empty + C::STAGES, *tfree = chain + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(tfree + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nitems = p.tilesA * p.tilesB * p.nsplit;
  if (tid == 0) {
    for (int i = 0; i < C::STAGES; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&chain[h], 1);
      tc::mbar_init(&tfree[h], 8);
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
    if (lane == 0) {  // loads: A digit t into plane t, B digit u into block T - 1 - u
      long g = 0;     // stages issued by this CTA
      for (int item = blockIdx.x; item < nitems && !fail; item += gridDim.x) {
        const OzItem it = oz_item(p, item);
        for (int i = 0; i < it.n; ++i, ++g) {
          const int st = (int)(g % C::STAGES);
          const long k = g / C::STAGES;
          if (k > 0 && !tc::mbar_wait(&empty[st], (uint32_t)((k - 1) & 1), kWaitLimit)) {
            fail = true;
            break;
          }
          unsigned char *S = sm + st * C::SB;
          const int kx = (it.c0 + i) * OZ_KS;
          mbar_expect_tx(&full[st], (uint32_t)C::SB);
#pragma unroll
          for (int t = 0; t < T; ++t) tma_load3d(S + t * C::AB, &mA, kx, it.a0, t, &full[st]);
#pragma unroll
          for (int u = 0; u < T; ++u) tma_load3d(S + T * C::AB + (T - 1 - u) * C::BB, &mB, kx, it.b0, u, &full[st]);
        }
      }
      // every copy issued lands before the block's shared memory goes away
      for (long i = max(0L, g - C::STAGES); i < g; ++i)
        if (!tc::mbar_wait(&full[i % C::STAGES], (uint32_t)((i / C::STAGES) & 1), kWaitLimit)) fail = true;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMAs
      long g = 0;     // stages consumed
      int q0 = 0;     // chains started by earlier items
      for (int item = blockIdx.x; item < nitems && !fail; item += gridDim.x) {
        const OzItem it = oz_item(p, item);
        for (int i = 0; i < it.n; ++i, ++g) {
          const int st = (int)(g % C::STAGES), q = q0 + i / OZ_CHAIN, first = (i % OZ_CHAIN) == 0;
          const long k = g / C::STAGES;
          if (first && q >= 2 && !tc::mbar_wait(&tfree[q & 1], ((q - 2) >> 1) & 1, kWaitLimit)) {
            fail = true;
            break;
          }
          if (!tc::mbar_wait(&full[st], (uint32_t)(k & 1), kWaitLimit)) {
            fail = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t base = tc::smem_u32(sm + st * C::SB);
          const uint32_t acc = tmem + (uint32_t)((q & 1) * 256);
#pragma unroll
          for (int ks = 0; ks < OZ_KS / 16; ++ks)
#pragma unroll
            for (int t = 0; t < T; ++t)
              mma_bf16(acc, tc::desc_sw64(base + t * C::AB + 32 * ks), tc::desc_sw64(base + T * C::AB + t * C::BB + 32 * ks),
                       idesc_bf16(OZ_M, (T - t) * OZ_NB), (first && ks == 0 && t == 0) ? 0u : 1u);
          tc::mma_commit(&empty[st]);
          if ((i % OZ_CHAIN) == OZ_CHAIN - 1 || i == it.n - 1) tc::mma_commit(&chain[q & 1]);
        }
        q0 += (it.n + OZ_CHAIN - 1) / OZ_CHAIN;
      }
      if (g > 0 && !tc::mbar_wait(&empty[(g - 1) % C::STAGES], (uint32_t)(((g - 1) / C::STAGES) & 1), kWaitLimit))
        fail = true;  // the MMAs issued have finished with TMEM and shared memory
    }
  } else if (warp >= 4) {  // chains out of TMEM; each item's result after its last chain
    const int qd = warp & 3, h = (warp - 4) >> 2;
    const int ra = 32 * qd + lane;  // tile row (TMEM lane)
    int q0 = 0;
    for (int item = blockIdx.x; item < nitems && !fail; item += gridDim.x) {
      const OzItem it = oz_item(p, item);
      const int nchains = (it.n + OZ_CHAIN - 1) / OZ_CHAIN;
      int ia[4][16];
      float fa[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        ia[0][c] = ia[1][c] = ia[2][c] = ia[3][c] = 0;
        fa[c] = 0.f;
      }
      for (int cc = 0; cc < nchains; ++cc) {
        const int q = q0 + cc;
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&chain[q & 1], (q >> 1) & 1, kWaitLimit))) {
          fail = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t base = tmem + (uint32_t)((q & 1) * 256) + ((uint32_t)(32 * qd) << 16) + (uint32_t)(16 * h);
#pragma unroll
        for (int b = 0; b < T; ++b) {
          constexpr float r7 = 1.0f / 128.0f;
          const int gidx = T - 1 - b;
          float v[16];
          tc::tmem_ld16(base + (uint32_t)(b * OZ_NB), v);
          if (gidx <= 3) {
#pragma unroll
            for (int c = 0; c < 16; ++c) ia[gidx][c] += __float2int_rn(v[c]);
          } else {
            float sc = 1.f;
#pragma unroll
            for (int e = 0; e < gidx; ++e) sc *= r7;
#pragma unroll
            for (int c = 0; c < 16; ++c) fa[c] = __fmaf_rn(v[c], sc, fa[c]);
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tfree[q & 1]);
      }
      q0 += nchains;
      const int a = it.a0 + ra;
      if (fail || a >= p.rowsA) continue;
      const int ea = p.eA[a];
      if constexpr (EPI == OZ_GRAM) {
        double *o = p.out + (size_t)it.z * p.split_stride + (size_t)a * p.ldo;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int b = it.b0 + 16 * h + c;
          if (b < p.rowsB) {
            const double v = (double)ia[0][c] + 0x1p-7 * (double)ia[1][c] + 0x1p-14 * (double)ia[2][c] + 0x1p-21 * (double)ia[3][c] +
                             (double)fa[c];
            o[b] = ldexp(v, ea + p.eB[b] - 14);
          }
        }
      } else {
        df64 *y = p.Y + (size_t)a * p.ldy;
        const int bb = it.b0 + 16 * h;
        df64 old[16];  // every load in flight before the arithmetic
#pragma unroll
        for (int c = 0; c < 16; ++c) old[c] = (p.c0 != 0.f && bb + c < p.rowsB) ? y[bb + c] : df64(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int b = bb + c;
          if (b < p.rowsB) {
            df64 s = df_of_int(ia[0][c]);
            const df64 t1 = df_of_int(ia[1][c]), t2 = df_of_int(ia[2][c]), t3 = df_of_int(ia[3][c]);
            s = s + df64(t1.hi * 0x1p-7f, t1.lo * 0x1p-7f);
            s = s + df64(t2.hi * 0x1p-14f, t2.lo * 0x1p-14f);
            s = s + df64(t3.hi * 0x1p-21f, t3.lo * 0x1p-21f);
            s = s + df64(fa[c], 0.f);
            const int e = ea + p.eB[b] - 14;
            s = df64(ldexpf(s.hi, e), ldexpf(s.lo, e));
            if (p.c0 != 0.f) s = s + (p.c0 > 0.f ? old[c] : -old[c]);
            y[b] = s;
          }
        }
      }
    }
  }
  fail = __syncthreads_or(fail);
  if (fail && tid == 0) atomicExch(p.err, 1);
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------------
// slicing

// balanced base-128 digits of an integer |I| <= 2^(7T): d[T-1] .. d[1] in [-64, 63], d[0] the rest
template <int T> __device__ __forceinline__ void oz_digits(long long I, float (&d)[T]) {
#pragma unroll
  for (int t = T - 1; t >= 1; --t) {
    const long long m = ((I + 64) & 127) - 64;
    d[t] = (float)m;
    I = (I - m) >> 7;
  }
  d[0] = (float)I;
}

__device__ __forceinline__ int oz_exponent(float m) { return m > 0.f ? ilogbf(m) + 1 : 0; }
__device__ __forceinline__ int oz_exponent(double m) { return m > 0.0 ? ilogb(m) + 1 : 0; }

// block-wide maximum of one value per thread (blockDim.x = 256); valid in every thread
template <typename V> __device__ V block_max256(V v) {
  __shared__ V red[8];
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  V r = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) r = max(r, red[w]);
  return r;
}

__device__ __forceinline__ void put_bf16x2(uint16_t *dst, float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  *reinterpret_cast<__nv_bfloat162 *>(dst) = v;
}

// digits of the rows of a complex matrix (K = 2 N_int real values per row, src[r][ld] complex),
// times the Gamma-point weights (1 on the first len0 elements, 2 on the rest) when weighted;
// one block of 256 threads per row, four elements per thread and iteration with their loads
// issued together. dig: [T][rows][kpad], ex: [rows].
template <int T>
__global__ void __launch_bounds__(256) k_oz_rows_df(const cplx<df64> *__restrict__ src, int ld, int nint, int len0, bool weighted,
                                                    uint16_t *__restrict__ dig, int kpad, size_t plane, int *__restrict__ ex) {
  constexpr int U = 4;
  const int r = blockIdx.x;
  const cplx<df64> *row = src + (size_t)r * ld;
  const cplx<df64> zero = mkc<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
  float m = 0.f;
  for (int e0 = threadIdx.x; e0 < nint; e0 += 256 * U) {
    cplx<df64> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = e0 + 256 * u < nint ? row[e0 + 256 * u] : zero;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float w = (weighted && e0 + 256 * u >= len0) ? 2.f : 1.f;
      m = fmaxf(m, w * fmaxf(fabsf(v[u].x.hi), fabsf(v[u].y.hi)));
    }
  }
  m = block_max256(m);
  const int E = oz_exponent(m);
  if (threadIdx.x == 0) ex[r] = E;
  const int sh = 7 * T - E;
  for (int e0 = threadIdx.x; e0 < nint; e0 += 256 * U) {
    cplx<df64> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = e0 + 256 * u < nint ? row[e0 + 256 * u] : zero;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + 256 * u;
      if (e >= nint) break;
      const int sw = sh + ((weighted && e >= len0) ? 1 : 0);
      const long long Ix = __float2ll_rn(ldexpf(v[u].x.hi, sw)) + __float2ll_rn(ldexpf(v[u].x.lo, sw));
      const long long Iy = __float2ll_rn(ldexpf(v[u].y.hi, sw)) + __float2ll_rn(ldexpf(v[u].y.lo, sw));
      float dx[T], dy[T];
      oz_digits<T>(Ix, dx);
      oz_digits<T>(Iy, dy);
#pragma unroll
      for (int t = 0; t < T; ++t) put_bf16x2(dig + t * plane + (size_t)r * kpad + 2 * e, dx[t], dy[t]);
    }
  }
}

// the same from FP64 rows (the projectors and orbitals, once per context)
template <int T>
__global__ void __launch_bounds__(256) k_oz_rows_f64(const cplx<double> *__restrict__ src, int ld, int nint, int len0, bool weighted,
                                                     uint16_t *__restrict__ dig, int kpad, size_t plane, int *__restrict__ ex) {
  const int r = blockIdx.x;
  const cplx<double> *row = src + (size_t)r * ld;
  double m = 0.0;
  for (int e = threadIdx.x; e < nint; e += 256) {
    const cplx<double> v = row[e];
    const double w = (weighted && e >= len0) ? 2.0 : 1.0;
    m = fmax(m, w * fmax(fabs(v.x), fabs(v.y)));
  }
  m = block_max256(m);
  const int E = oz_exponent(m);
  if (threadIdx.x == 0) ex[r] = E;
  for (int e = threadIdx.x; e < nint; e += 256) {
    const cplx<double> v = row[e];
    const int sw = 7 * T - E + ((weighted && e >= len0) ? 1 : 0);
    float dx[T], dy[T];
    oz_digits<T>(__double2ll_rn(ldexp(v.x, sw)), dx);
    oz_digits<T>(__double2ll_rn(ldexp(v.y, sw)), dy);
#pragma unroll
    for (int t = 0; t < T; ++t) put_bf16x2(dig + t * plane + (size_t)r * kpad + 2 * e, dx[t], dy[t]);
  }
}

// digits of the transpose of an FP64 matrix src[j][c] (j < nj rows, c < ncol columns, row stride
// lds), each source row scaled by d[j] when d is given: output row c has K = nj values (over j)
// and its own exponent. Blocks of 32 columns x 8 row lanes; dig: [T][ncol][kpad], ex: [ncol].
template <int T>
__global__ void __launch_bounds__(256) k_oz_cols(const double *__restrict__ src, size_t lds, int nj, int ncol, const double *__restrict__ d,
                                                 uint16_t *__restrict__ dig, int kpad, size_t plane, int *__restrict__ ex) {
  __shared__ double red[8][33];
  __shared__ float tile[T][32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c0 = blockIdx.x * 32, c = c0 + tx;
  double m = 0.0;
  if (c < ncol)
    for (int j = ty; j < nj; j += 8) m = fmax(m, fabs(src[(size_t)j * lds + c] * (d ? d[j] : 1.0)));
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w][tx]);
    red[0][tx] = (double)oz_exponent(m);
    if (c < ncol) ex[c] = oz_exponent(m);
  }
  __syncthreads();
  const int E = (int)red[0][tx];
  for (int j0 = 0; j0 < nj; j0 += 32) {
    // rows j0 + ty + 8 i: thread (tx, ty) makes the digits of column c, then writes them transposed
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int jj = ty + 8 * i, j = j0 + jj;
      float dd[T];
      double v = 0.0;
      if (c < ncol && j < nj) v = src[(size_t)j * lds + c] * (d ? d[j] : 1.0);
      oz_digits<T>(__double2ll_rn(ldexp(v, 7 * T - E)), dd);
#pragma unroll
      for (int t = 0; t < T; ++t) tile[t][tx][jj] = dd[t];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int cc = ty + 8 * i, col = c0 + cc, j = j0 + tx;
      if (col < ncol && j < nj) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const __nv_bfloat16 b = __float2bfloat16_rn(tile[t][cc][tx]);
          dig[t * plane + (size_t)col * kpad + j] = __bfloat16_as_ushort(b);
        }
      }
    }
    __syncthreads();
  }
}

// out[j][s] (row stride ldo) = sum of the split partials work[k][j][s] (row stride nb)
__global__ void k_oz_sum_splits(const double *__restrict__ work, int nsplit, size_t stride, double *__restrict__ out, int na, int nb,
                                int ldo) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)na * nb) return;
  const int j = (int)(t / nb), s = (int)(t % nb);
  double a = 0.0;
  for (int k = 0; k < nsplit; ++k) a += work[k * stride + (size_t)j * nb + s];
  out[(size_t)j * ldo + s] = a;
}

// rows of K bf16 digits, T planes ([T][rows][kpad]), read in boxes of 32 x box_rows into
// 64-byte swizzled shared memory; reads past K or the last row return zeros
CUtensorMap digit_map(const uint16_t *base, int K, int rows, int kpad, size_t plane, int box_rows, int T) {
  CUtensorMap m;
  const cuuint64_t dim[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)T};
  const cuuint64_t stride[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)plane * 2};
  const cuuint32_t box[3] = {(cuuint32_t)OZ_KS, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = tmap_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t *>(base), dim, stride, box, es,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw ApiFailure(WDF_EINVAL, "tensor map encoding failed (" + std::to_string((int)r) + ")");
  return m;
}

int num_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  return nsm;
}

template <int T, int EPI>
void run_gemm(const OzMat &A, const OzMat &B, int K, OzArgs p, double *work, size_t work_cap, cudaStream_t st) {
  p.rowsA = A.rows;
  p.rowsB = B.rows;
  p.eA = A.ex;
  p.eB = B.ex;
  p.tilesA = (A.rows + OZ_M - 1) / OZ_M;
  p.tilesB = (B.rows + OZ_NB - 1) / OZ_NB;
  p.nst = (K + OZ_KS - 1) / OZ_KS;
  // K splits: enough CTAs for the SMs, and at most OZ_MAXCHAIN chains per split
  const int tiles = p.tilesA * p.tilesB, nsm = num_sms();
  int nsplit = std::max(1, (p.nst + OZ_CHAIN * OZ_MAXCHAIN - 1) / (OZ_CHAIN * OZ_MAXCHAIN));
  if (EPI == OZ_GRAM)
    while (tiles * nsplit < nsm && p.nst / (nsplit + 1) >= 4 * OZ_CHAIN) ++nsplit;
  p.per = (p.nst + nsplit - 1) / nsplit;
  nsplit = std::max(1, (p.nst + p.per - 1) / p.per);
  double *final_out = p.out;
  const int final_ldo = p.ldo;
  if (EPI == OZ_GRAM && nsplit > 1) {
    if ((size_t)nsplit * A.rows * B.rows > work_cap) throw ApiFailure(WDF_EINVAL, "tensor-core projection workspace too small");
    p.out = work;
    p.ldo = B.rows;
    p.split_stride = (size_t)A.rows * B.rows;
  } else {
    p.split_stride = 0;
  }
  if (EPI == OZ_LINCOMB && nsplit > 1) throw ApiFailure(WDF_EINVAL, "linear combination over too many rows of U");
  p.groupA = EPI == OZ_GRAM ? p.tilesA : std::min(p.tilesA, 16);
  const CUtensorMap mA = digit_map(A.dig, K, A.rows, A.kpad, A.plane, OZ_M, T);
  const CUtensorMap mB = digit_map(B.dig, K, B.rows, B.kpad, B.plane, OZ_NB, T);
  p.nsplit = nsplit;
  const int grid = std::min(tiles * nsplit, nsm);  // persistent: one CTA per SM
  launch(EPI == OZ_GRAM ? "gram" : "lincomb", 64, k_oz_gemm<T, EPI>, dim3(grid), dim3(OZ_THREADS), oz_smem<T>(), st, mA, mB, p);
  WDF_CUDA_TRY(cudaGetLastError());
  if (EPI == OZ_GRAM && nsplit > 1) {
    launch("gram_sum", 0, k_oz_sum_splits, dim3((unsigned)(((size_t)A.rows * B.rows + 255) / 256)), dim3(256), 0, st, (const double *)work,
           nsplit, p.split_stride, final_out, A.rows, B.rows, final_ldo);
    WDF_CUDA_TRY(cudaGetLastError());
  }
}

}  // namespace

bool oz_enabled() {
  static const bool on = std::getenv("WDF_NO_OZ") == nullptr;
  return on && tc_enabled();
}

int oz_kpad(int K) { return ((K + OZ_KS - 1) / OZ_KS) * OZ_KS; }

void set_oz_limits() {
  raise_smem_limit(k_oz_gemm<OZ_DIGITS, OZ_GRAM>, oz_smem<OZ_DIGITS>());
  raise_smem_limit(k_oz_gemm<OZ_DIGITS, OZ_LINCOMB>, oz_smem<OZ_DIGITS>());
}

void launch_oz_rows_df(const Geo &g, const cplx<df64> *src, int rows, bool weighted, const OzMat &out, cudaStream_t st) {
  if (rows <= 0) return;
  launch("oz_slice", 64, k_oz_rows_df<OZ_DIGITS>, dim3(rows), dim3(256), 0, st, src, g.ld, g.nint, g.len0, weighted, out.dig, out.kpad,
         out.plane, out.ex);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_oz_rows_f64(const Geo &g, const cplx<double> *src, int rows, bool weighted, const OzMat &out, cudaStream_t st) {
  if (rows <= 0) return;
  launch("oz_slice", 64, k_oz_rows_f64<OZ_DIGITS>, dim3(rows), dim3(256), 0, st, src, g.ld, g.nint, g.len0, weighted, out.dig, out.kpad,
         out.plane, out.ex);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_oz_cols(const double *src, size_t lds, int nj, int ncol, const double *d, const OzMat &out, cudaStream_t st) {
  if (ncol <= 0) return;
  launch("oz_slice", 64, k_oz_cols<OZ_DIGITS>, dim3((ncol + 31) / 32), dim3(256), 0, st, src, lds, nj, ncol, d, out.dig, out.kpad,
         out.plane, out.ex);
  WDF_CUDA_TRY(cudaGetLastError());
}

size_t oz_gram_work_doubles(int na, int nb, int K) {
  const int nst = (K + OZ_KS - 1) / OZ_KS;
  const int tiles = ((na + OZ_M - 1) / OZ_M) * ((nb + OZ_NB - 1) / OZ_NB);
  int nsplit = std::max(1, (nst + OZ_CHAIN * OZ_MAXCHAIN - 1) / (OZ_CHAIN * OZ_MAXCHAIN));
  while (tiles * nsplit < num_sms() && nst / (nsplit + 1) >= 4 * OZ_CHAIN) ++nsplit;
  return nsplit > 1 ? (size_t)nsplit * na * nb : 0;
}

void launch_oz_gram(const OzMat &U, const OzMat &X, int K, double *out, int ldo, double *work, size_t work_cap, int *err, cudaStream_t st) {
  if (U.rows <= 0 || X.rows <= 0) return;
  OzArgs p{};
  p.out = out;
  p.ldo = ldo;
  p.err = err;
  run_gemm<OZ_DIGITS, OZ_GRAM>(U, X, K, p, work, work_cap, st);
}

void launch_oz_lincomb(const OzMat &C, const OzMat &Ut, int K, df64 *Y, size_t ldy, float c0, int *err, cudaStream_t st) {
  if (C.rows <= 0 || Ut.rows <= 0) return;
  OzArgs p{};
  p.Y = Y;
  p.ldy = ldy;
  p.c0 = c0;
  p.err = err;
  run_gemm<OZ_DIGITS, OZ_LINCOMB>(C, Ut, K, p, nullptr, 0, st);
}

}  // namespace wdf

// Tensor-core (tcgen05, kind::tf32) forms of the two dense products of the FP32 inner CG:
//   gram:    S[j][s] = sum_e w_e Re(conj(U_j[e]) X_s[e])       (projections on [beta; psi])
//   lincomb: Y_s = c0 Y_s + sum_j U_j S[j][s] d_j               (KB term and alpha P shift)
// Complex vectors are read as real rows of 2 N_int values, so both are real GEMMs with K-major
// operands. FP32 accuracy from TF32 units by the three-term split a b ~ a_h b_h + a_h b_l + a_l b_h
// with a_h the upper 19 bits of a and a_l = a - a_h (the dropped a_l b_l is ~2^-22 |a b|).
// Operand tiles are staged through registers (the low parts and the zero padding are made on
// the way) into 128-byte-swizzled shared memory, two stages deep; one thread issues the MMAs and
// commits them to the stage's mbarrier; accumulators sit in TMEM and the epilogue reads them with
// tcgen05.ld. Every mbarrier wait is bounded: on expiry the kernel raises a flag, waits (bounded)
// for what it issued, frees its TMEM and returns.
#include <cstdlib>

#include "engine.cuh"
#include "tc.cuh"

namespace wdf {

namespace {

constexpr int TM = 128;              // MMA M: solves per tile
constexpr int TK = 32;               // K values per stage (one 128-byte row)
constexpr int XB = TM * 128;         // bytes of a 128-row operand tile
constexpr long kWaitLimit = 1L << 26;  // polls of an mbarrier before giving up
// chunks per FP32 accumulation chain of the Gram: longer chains lose accuracy (the sums run over
// 2 N_int products), so every kPromote chunks the partial sums move into the FP64 output
constexpr int kPromote = 32;

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return (unsigned char *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// stage a 16-byte piece (hi and lo) into swizzled tiles
__device__ __forceinline__ void put(unsigned char *hi, unsigned char *lo, int row, int q, float4 v) {
  const int o = tc::swz_off(row, q);
  *reinterpret_cast<float4 *>(hi + o) = v;
  *reinterpret_cast<float4 *>(lo + o) = make_float4(tc::tf32_low(v.x), tc::tf32_low(v.y), tc::tf32_low(v.z), tc::tf32_low(v.w));
}

// element f .. f+3 of a row, zero at and beyond kf
__device__ __forceinline__ float4 load_masked(const float *row, int f, int kf) {
  if (f + 3 < kf) return *reinterpret_cast<const float4 *>(row + f);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (f < kf) v.x = row[f];
  if (f + 1 < kf) v.y = row[f + 1];
  if (f + 2 < kf) v.z = row[f + 2];
  return v;
}

// S (+ split partials) = U_w X^T; grid (solve tiles, splits), 256 threads. The operands of chunk
// i + 1 are loaded into registers while the MMAs of chunk i run, so global latency overlaps them.
constexpr int UPT = 8;  // U pieces per thread and operand part at most (256 rows x 8 pieces / 256 threads)

// blockIdx.z picks a chunk of at most kGramRows rows of U (rows z kGramRows ...): a CTA holds the
// accumulators of 128 solves x one chunk in TMEM, so U of any height runs in chunks.
constexpr int kGramRows = 256;

__global__ void __launch_bounds__(256, 1) k_gram_tc(Geo g, const float *__restrict__ X, int nb, const float *__restrict__ Uhi,
                                                    const float *__restrict__ Ulo, int na_all, double *__restrict__ out, int ldo,
                                                    int ch_per_split, size_t split_stride, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = align1024(smraw);
  const int j0 = blockIdx.z * kGramRows;
  const int na = min(kGramRows, na_all - j0), nu = ((na + 31) / 32) * 32;
  Uhi += (size_t)j0 * 2 * g.ld;
  Ulo += (size_t)j0 * 2 * g.ld;
  out += (size_t)j0 * ldo;
  const int UB = nu * 128, SB = 2 * XB + 2 * UB;  // the launch sizes shared memory for the largest chunk
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * SB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + 2 * SB + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * TM;
  const int kf = 2 * g.nint, ldf = 2 * g.ld;
  const int nch = (kf + TK - 1) / TK;
  const int c0 = blockIdx.y * ch_per_split, c1 = min(nch, c0 + ch_per_split);
  const int upt = (nu * 8) / 256;  // nu is a multiple of 32, so whole pieces per thread
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t idesc = tc::idesc_tf32(TM, nu);
  // accumulation chains of kPromote chunks alternate between the two TMEM halves; a finished
  // chain is added into the FP64 output while the next one accumulates in the other half
  const int qd = warp & 3, hh = warp >> 2, orow = 32 * qd + lane, osol = s0 + orow;
  double *o = out + (size_t)blockIdx.y * split_stride;
  auto promote = [&](int p) {  // the first chain stores, later chains add
    tc::fence_after_sync();
    const uint32_t base = tmem + (uint32_t)((p & 1) * 256);
    const int halfc = nu / 2;
    for (int cg = 0; cg < halfc; cg += 16) {
      const int col = hh * halfc + cg;
      float v[16];
      tc::tmem_ld16(base + ((uint32_t)(32 * qd) << 16) + (uint32_t)col, v);
      if (osol < nb)
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (col + k < na) {
            double *d = o + (size_t)(col + k) * ldo + osol;
            *d = p == 0 ? (double)v[k] : *d + (double)v[k];
          }
    }
    tc::fence_before_sync();
  };
  int promoted = 0;
  float4 rx[4], rh[UPT], rl[UPT];
  auto fetch = [&](int c) {
    const int f0 = c * TK;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = tid + 256 * u, row = t >> 3, q = t & 7;
      rx[u] = (s0 + row < nb) ? load_masked(X + (size_t)(s0 + row) * ldf, f0 + 4 * q, kf) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const int t = tid + 256 * u, row = t >> 3, q = t & 7;
      rh[u] = rl[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < upt && row < na) {
        rh[u] = *reinterpret_cast<const float4 *>(Uhi + (size_t)row * ldf + f0 + 4 * q);
        rl[u] = *reinterpret_cast<const float4 *>(Ulo + (size_t)row * ldf + f0 + 4 * q);
      }
    }
  };
  if (c0 < c1) fetch(c0);
  int issued = 0;
  bool ok = true;
  for (int c = c0; c < c1; ++c) {
    const int i = c - c0, st = i & 1;
    unsigned char *S = sm + st * SB;
    if (i >= 2) ok = __syncthreads_and(ok && tc::mbar_wait(&bar[st], ((i - 2) >> 1) & 1, kWaitLimit));
    if (!ok) break;
    if (i >= 2 && (i - 2) % kPromote == kPromote - 1) {  // chunk i - 2 closed a chain: its MMAs are done
      promote((i - 2) / kPromote);
      promoted = (i - 2) / kPromote + 1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = tid + 256 * u;
      put(S, S + XB, t >> 3, t & 7, rx[u]);
    }
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const int t = tid + 256 * u;
      if (u < upt) {
        const int o = tc::swz_off(t >> 3, t & 7);
        *reinterpret_cast<float4 *>(S + 2 * XB + o) = rh[u];
        *reinterpret_cast<float4 *>(S + 2 * XB + UB + o) = rl[u];
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t base = tc::smem_u32(S);
      const uint32_t acc = tmem + (uint32_t)(((i / kPromote) & 1) * 256);
      const int first = i % kPromote;
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const uint32_t a = base + (term == 2 ? XB : 0), b = base + 2 * XB + (term == 1 ? UB : 0);
#pragma unroll
        for (int ks = 0; ks < TK / 8; ++ks)
          tc::mma_tf32(acc, tc::desc_sw128(a + 32 * ks), tc::desc_sw128(b + 32 * ks), idesc, (first | term | ks) ? 1u : 0u);
      }
      tc::mma_commit(&bar[st]);
    }
    ++issued;
    if (c + 1 < c1) fetch(c + 1);  // in flight while the MMAs run
  }
  // the last commit covers every MMA issued
  bool done = issued == 0 ? true : tc::mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitLimit);
  done = __syncthreads_and(done) && ok && issued == c1 - c0;
  if (done) {
    if (issued == 0) {  // an empty K range still owns its part of the output
      if (osol < nb)
        for (int col = hh * (nu / 2); col < (hh + 1) * (nu / 2) && col < na; ++col) o[(size_t)col * ldo + osol] = 0.0;
    }
    for (int p = promoted; p * kPromote < issued; ++p) promote(p);  // the chains still in TMEM (at most two)
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
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
// grid (solve tiles, 256-value tiles), 256 threads. Operands of the next K chunk are fetched into
// registers while the MMAs run; the finished tile goes TMEM -> shared memory, then each warp
// updates whole rows of Y with coalesced accesses and reduces its row's partial inner product.
constexpr int DP = 260;  // shared row pitch of the result tile (floats): conflict-free float4 stores

__global__ void __launch_bounds__(256, 1) k_lincomb_tc(Geo g, float *__restrict__ Y, int ny, const float *__restrict__ Chi,
                                                       const float *__restrict__ Clo, int kp, const float *__restrict__ Uthi,
                                                       const float *__restrict__ Utlo, float c0, const float *__restrict__ P,
                                                       double *__restrict__ part, int nchunk, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = align1024(smraw);
  constexpr int TN = 256, BB = TN * 128, SB = 2 * XB + 2 * BB;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * SB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + 2 * SB + 16);
  float *D = reinterpret_cast<float *>(sm);  // result tile [128][DP], over the operand stages
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * TM, f0 = blockIdx.y * TN;
  const int kf = 2 * g.nint, ldf = 2 * g.ld;
  const int nkc = kp / TK;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(slot, 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t idesc = tc::idesc_tf32(TM, TN);
  float4 ah[4], al[4], bh[8], bl[8];
  auto fetch = [&](int i) {
    const int k0 = i * TK;
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // coefficients: 128 solve rows x 8 pieces (hi, lo precomputed)
      const int t = tid + 256 * u, row = t >> 3, q = t & 7;
      ah[u] = al[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s0 + row < ny) {
        ah[u] = *reinterpret_cast<const float4 *>(Chi + (size_t)(s0 + row) * kp + k0 + 4 * q);
        al[u] = *reinterpret_cast<const float4 *>(Clo + (size_t)(s0 + row) * kp + k0 + 4 * q);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {  // U transposed: 256 value rows x 8 pieces
      const int t = tid + 256 * u, row = t >> 3, q = t & 7;
      bh[u] = bl[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f0 + row < kf) {
        bh[u] = *reinterpret_cast<const float4 *>(Uthi + (size_t)(f0 + row) * kp + k0 + 4 * q);
        bl[u] = *reinterpret_cast<const float4 *>(Utlo + (size_t)(f0 + row) * kp + k0 + 4 * q);
      }
    }
  };
  fetch(0);
  int issued = 0;
  bool ok = true;
  for (int i = 0; i < nkc; ++i) {
    const int st = i & 1;
    unsigned char *S = sm + st * SB;
    if (i >= 2) ok = __syncthreads_and(ok && tc::mbar_wait(&bar[st], ((i - 2) >> 1) & 1, kWaitLimit));
    if (!ok) break;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = tid + 256 * u, o = tc::swz_off(t >> 3, t & 7);
      *reinterpret_cast<float4 *>(S + o) = ah[u];
      *reinterpret_cast<float4 *>(S + XB + o) = al[u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = tid + 256 * u, o = tc::swz_off(t >> 3, t & 7);
      *reinterpret_cast<float4 *>(S + 2 * XB + o) = bh[u];
      *reinterpret_cast<float4 *>(S + 2 * XB + BB + o) = bl[u];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t base = tc::smem_u32(S);
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const uint32_t a = base + (term == 2 ? XB : 0), b = base + 2 * XB + (term == 1 ? BB : 0);
#pragma unroll
        for (int ks = 0; ks < TK / 8; ++ks)
          tc::mma_tf32(tmem, tc::desc_sw128(a + 32 * ks), tc::desc_sw128(b + 32 * ks), idesc, (i | term | ks) ? 1u : 0u);
      }
      tc::mma_commit(&bar[st]);
    }
    ++issued;
    if (i + 1 < nkc) fetch(i + 1);
  }
  bool done = issued == 0 ? true : tc::mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kWaitLimit);
  done = __syncthreads_and(done) && ok && issued == nkc;
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

size_t gram_tc_smem(int nu) { return 1024 + 2 * (size_t)(2 * XB + 2 * nu * 128) + 64; }
size_t lincomb_tc_smem() { return 1024 + 2 * (size_t)(2 * XB + 2 * 256 * 128) + 64; }

}  // namespace

bool tc_enabled() {
  static const bool on = std::getenv("WDF_NO_TC") == nullptr;
  return on;
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
// choose the split count (at most nch / 8, so that each CTA keeps a pipeline of >= 8 chunks)
// that minimises waves x (chunks per CTA + 6), the 6 standing for a CTA's partial-sum write
// (128 x 192 doubles, about the bytes of a dozen X chunks, written without waiting), the smaller
// count on ties (fewer partial sums to add)
static int gram_tc_splits(int nch, int tiles) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  const int smax = std::max(1, std::min(nch / 8, 4 * ((nsm + tiles - 1) / tiles)));
  long best = -1;
  int bs = 1;
  for (int sp = 1; sp <= smax; ++sp) {
    const long waves = ((long)tiles * sp + nsm - 1) / nsm, per = (nch + sp - 1) / sp;
    const long cost = waves * (per + 6);
    if (best < 0 || cost < best) {
      best = cost;
      bs = sp;
    }
  }
  return bs;
}

size_t gram_tc_work_doubles(const Geo &g, int na, int nb) {
  const int nch = (2 * g.nint + TK - 1) / TK;
  const int tiles = ((nb + TM - 1) / TM) * ((na + kGramRows - 1) / kGramRows);
  const int nsplit = gram_tc_splits(nch, tiles);
  return nsplit > 1 ? (size_t)nsplit * na * nb : 0;
}

void launch_gram_tc(const Geo &g, const float *X, int nb, const float *uwh, const float *uwl, int na, double *out, double *work,
                    size_t work_cap, int *err, cudaStream_t st) {
  if (nb <= 0 || na <= 0) return;
  const int nmc = (na + kGramRows - 1) / kGramRows;
  const int nu = tc_rows(std::min(na, kGramRows));
  const int nch = (2 * g.nint + TK - 1) / TK;
  const int tiles = (nb + TM - 1) / TM;
  int nsplit = gram_tc_splits(nch, tiles * nmc);
  if ((size_t)nsplit * na * nb > work_cap) nsplit = 1;
  const int per = (nch + nsplit - 1) / nsplit;
  nsplit = (nch + per - 1) / per;
  if (nsplit == 1) {
    launch("gram", 32, k_gram_tc, dim3(tiles, 1, nmc), dim3(256), gram_tc_smem(nu), st, g, X, nb, uwh, uwl, na, out, nb, per, (size_t)0,
           err);
  } else {
    const size_t stride = (size_t)na * nb;
    launch("gram", 32, k_gram_tc, dim3(tiles, nsplit, nmc), dim3(256), gram_tc_smem(nu), st, g, X, nb, uwh, uwl, na, work, nb, per,
           stride, err);
    WDF_CUDA_TRY(cudaGetLastError());
    launch("gram_sum", 0, k_tc_sum_splits, dim3((unsigned)(((size_t)na * nb + 255) / 256)), dim3(256), 0, st, (const double *)work,
           nsplit, stride, out, na, nb, nb);
  }
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_lincomb_tc(const Geo &g, float *Y, int ny, const double *S, int ldc, const double *d, int na, float *chi, float *clo,
                       const float *uth, const float *utl, float c0, const float *P, double *part, int *err, cudaStream_t st) {
  if (ny <= 0) return;
  const int kp = tc_rows(na);
  launch("lincomb", 32, k_tc_coef, dim3((ny + 31) / 32, (kp + 31) / 32), dim3(32, 8), 0, st, S, ldc, d, na, ny, kp, chi, clo);
  WDF_CUDA_TRY(cudaGetLastError());
  const int ntile = (2 * g.nint + 255) / 256;
  launch("lincomb", 32, k_lincomb_tc, dim3((ny + TM - 1) / TM, ntile), dim3(256), lincomb_tc_smem(), st, g, Y, ny, (const float *)chi,
         (const float *)clo, kp, uth, utl, c0, P, part, lincomb_dot_chunks(g), err);
  WDF_CUDA_TRY(cudaGetLastError());
}

}  // namespace wdf

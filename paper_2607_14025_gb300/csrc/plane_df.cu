// Double-float plane kernel for 64 x 64 planes: the V_loc product of the FP64-class residuals,
// the right-hand-side product psi_v dV and the orbital sum of the density response.
//
// Same transforms as k_plane_fast (Stockham radix 8 x 8 along n2 for the occupied columns and
// along n1 for every row, natural order in and out), organised for code size: a double-float
// radix-8 butterfly is ~900 FP32 instructions, and the unrolled passes of the general kernel
// (eight passes, two tasks per thread) put ~16 of them in one kernel, far beyond the instruction
// cache. Here 512 threads each run one radix-8 task per pass, and the eight passes of a plane
// (n2 inverse A and B, n1 inverse A and B, n1 forward A and B, n2 forward A and B) are a runtime
// loop over one task body per direction. Pass A (stride 1) reads elements j + 8 r of its line and
// writes 8 j + r; pass B multiplies element r by w^(r j) (the conjugate in the forward direction),
// reads and writes j + 8 r. The n1 inverse transform ends with elements j + 8 r of row t % 64 in
// registers, which is where the product with V_loc (or the orbital sum) happens and where the n1
// forward transform starts. The V_loc and product forms fit 64 registers, so two blocks share an
// SM and one block's barriers do not idle it; the orbital-sum form holds a second register block
// (the running sum) and runs one block per SM.
#include <cstdlib>

#include "fft.cuh"
#include "kernels.cuh"
#include "stockham.cuh"

namespace wdf {
namespace {

constexpr int kN = 64;
constexpr int kP = kN + 1;  // tile pitch (odd: conflict-free rows and columns)
constexpr int kThreads = 512;
typedef cplx<df64> cd;

// one radix-8 Stockham task; `second` selects pass B (twiddles before the DFT)
__device__ __forceinline__ void df_task(cd (&v)[8], int j, bool second, int sg, const cd *tw) {
  if (second) {
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      cd w = tw[(r * j) & (kN - 1)];
      if (sg < 0) w.y = -w.y;
      v[r] = cmul<df64>(v[r], w);
    }
  }
  if (sg > 0) dft_reg<df64, 8, 1>(v);
  else dft_reg<df64, 8, -1>(v);
}

struct DfGeo {
  cd *tile;
  const cd *tw;
  const int *jidx;
  int xmax;
  bool col_on;  // this thread has a column task (t < 8 nx)
  int cj, cx;   // column task: butterfly and natural x of its column
  int rl, rj;   // row task: row and butterfly
};

__device__ __forceinline__ bool on_disk(int x, int xmax) { return x <= xmax || x >= kN - xmax; }

// phases ph0 .. ph1 - 1 of a plane: 0, 1 n2 inverse (phase 0 gathers from cbin); 2, 3 n1 inverse
// (phase 3 ends in registers and applies `mid`); 4, 5 n1 forward (phase 4 starts from registers);
// 6, 7 n2 forward (phase 7 scatters to cbout)
template <typename Mid>
__device__ __forceinline__ void df_phases(const DfGeo &d, int ph0, int ph1, cd (&v)[8], const cd *cbin, cd *cbout, Mid mid) {
#pragma unroll 1
  for (int ph = ph0; ph < ph1; ++ph) {
    const bool col = ph < 2 || ph >= 6;
    const bool on = col ? d.col_on : true;
    const int j = col ? d.cj : d.rj;
    const int sg = ph < 4 ? 1 : -1;
    const bool second = (ph & 1) != 0;
    if (on) {
      if (ph == 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int jj = __ldg(d.jidx + (j + 8 * r) * kN + d.cx);
          v[r] = jj >= 0 ? cbin[jj] : mkc<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
        }
      } else if (ph == 4) {
        // inputs already in registers
      } else if (col) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = d.tile[(j + 8 * r) * kP + d.cx];
      } else if (ph == 2) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int x = j + 8 * r;
          v[r] = on_disk(x, d.xmax) ? d.tile[d.rl * kP + x] : mkc<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = d.tile[d.rl * kP + j + 8 * r];
      }
      df_task(v, j, second, sg, d.tw);
    }
    if (ph == 3) {  // elements j + 8 r of row rl in registers
      mid(v);
      continue;
    }
    __syncthreads();  // every load of this in-place pass is done
    if (on) {
      if (ph == 7) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int jj = __ldg(d.jidx + (j + 8 * r) * kN + d.cx);
          if (jj >= 0) cbout[jj] = v[r];
        }
      } else if (col) {
#pragma unroll
        for (int r = 0; r < 8; ++r) d.tile[(second ? j + 8 * r : 8 * j + r) * kP + d.cx] = v[r];
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int x = second ? j + 8 * r : 8 * j + r;
          if (ph != 5 || on_disk(x, d.xmax)) d.tile[d.rl * kP + x] = v[r];  // the n2 passes read disk columns only
        }
      }
    }
    __syncthreads();
  }
}

template <int OP>
__global__ void __launch_bounds__(kThreads, OP == OP_ACCUM ? 1 : 2) k_plane_df(Geo g, const cd *__restrict__ twg, const int *__restrict__ jidx,
                                                         PlaneArgs<df64> pa) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cd *tw = reinterpret_cast<cd *>(smraw);
  cd *tile = tw + kN;
  int *xact = reinterpret_cast<int *>(tile + kN * kP);
  const int t = threadIdx.x;
  if (t < kN) tw[t] = twg[t];
  for (int i = t; i < g.nxact; i += kThreads) xact[i] = g.xactn[i];
  __syncthreads();
  const int nx = g.nxact, z = blockIdx.y;
  const size_t cbpair = (size_t)g.n3 * g.ldcb;
  constexpr size_t plane = (size_t)kN * kN;
  DfGeo d;
  d.tile = tile;
  d.tw = tw;
  d.jidx = jidx;
  d.xmax = g.xmax;
  d.col_on = t < 8 * nx;
  d.cj = d.col_on ? t / nx : 0;
  d.cx = d.col_on ? xact[t % nx] : 0;
  d.rl = t & (kN - 1);
  d.rj = t >> 6;
  cd v[8];
  if constexpr (OP == OP_VLOC) {
    const int q = blockIdx.x;
    cd *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    const df64 *vz = pa.field + (size_t)z * plane + (size_t)d.rl * kN + d.rj;
    df_phases(d, 0, 8, v, cbz, cbz, [&](cd(&w)[8]) {
#pragma unroll
      for (int r = 0; r < 8; ++r) w[r] = cscal<df64>(w[r], vz[8 * r]);
    });
  } else if constexpr (OP == OP_PROD_R2G) {
    // pair q = pp * nocc + v:  F(r) = psi_v(r) (dV_2pp + i dV_2pp+1)(r), row rl, elements rj + 8 r
    const int q = blockIdx.x;
    const int vo = q % pa.nocc, pp = q / pa.nocc;
    const size_t off = (size_t)z * plane + (size_t)d.rl * kN + d.rj;
    const df64 *psi = pa.field + (size_t)vo * g.n3 * plane + off;
    const cd *dv = pa.grid + (size_t)pp * g.n3 * plane + off;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = cscal<df64>(dv[8 * r], psi[8 * r]);
    cd *cbz = pa.cb + q * cbpair + (size_t)z * g.ldcb;
    df_phases(d, 4, 8, v, nullptr, cbz, [](cd(&)[8]) {});
  } else {  // OP_ACCUM: acc(r) = sum_v psi_v(r) G2R(cb[pp nocc + v]) in registers, then r -> G into cb2[pp]
    const int pp = blockIdx.x;
    cd acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = mkc<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
    const size_t off = (size_t)z * plane + (size_t)d.rl * kN + d.rj;
#pragma unroll 1
    for (int vo = 0; vo < pa.nocc; ++vo) {
      const cd *cbz = pa.cb + ((size_t)pp * pa.nocc + vo) * cbpair + (size_t)z * g.ldcb;
      const df64 *psi = pa.field + (size_t)vo * g.n3 * plane + off;
      df_phases(d, 0, 4, v, cbz, nullptr, [&](cd(&w)[8]) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const df64 s = psi[8 * r];
          acc[r].x += s * w[r].x;
          acc[r].y += s * w[r].y;
        }
      });
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = acc[r];
    cd *cbz = pa.cb2 + (size_t)pp * cbpair + (size_t)z * g.ldcb;
    df_phases(d, 4, 8, v, nullptr, cbz, [](cd(&)[8]) {});
  }
}

size_t df_smem(const Geo &g) { return sizeof(cd) * ((size_t)kN + (size_t)kN * kP) + sizeof(int) * (size_t)g.nxact; }

bool df_plane_enabled() {
  static const bool on = std::getenv("WDF_NO_DF_PLANE") == nullptr;
  return on;
}

}  // namespace

bool plane_df_available(const Geo &g, const int *jidx) {
  return df_plane_enabled() && jidx != nullptr && g.n1 == kN && g.n2 == kN && g.nxact >= 1 && g.nxact <= kN;
}

void set_plane_df_limits(const Geo &g) {
  if (g.n1 != kN || g.n2 != kN) return;
  const size_t sm = df_smem(g);
  raise_smem_limit(k_plane_df<OP_VLOC>, sm);
  raise_smem_limit(k_plane_df<OP_PROD_R2G>, sm);
  raise_smem_limit(k_plane_df<OP_ACCUM>, sm);
}

bool launch_plane_df(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st) {
  if (!plane_df_available(f.g, f.jidx) || nblk <= 0) return false;
  const dim3 grid(nblk, f.g.n3);
  const size_t sm = df_smem(f.g);
  switch (op) {
    case OP_VLOC: launch("plane_vloc", 48, k_plane_df<OP_VLOC>, grid, dim3(kThreads), sm, st, f.g, f.tw1, f.jidx, pa); break;
    case OP_PROD_R2G: launch("plane_prod", 48, k_plane_df<OP_PROD_R2G>, grid, dim3(kThreads), sm, st, f.g, f.tw1, f.jidx, pa); break;
    case OP_ACCUM: launch("plane_accum", 48, k_plane_df<OP_ACCUM>, grid, dim3(kThreads), sm, st, f.g, f.tw1, f.jidx, pa); break;
    default: return false;
  }
  WDF_CUDA_TRY(cudaGetLastError());
  return true;
}

}  // namespace wdf

// Launchers of the compile-time n3 transforms for a list of grid sizes (one instantiation per
// size, precision and epilogue). Each translation unit instantiates one precision and one size
// list (the build compiles them in parallel): zpass_fast_*.cu the common sizes, zpass_more_*.cu
// the further sizes of cubic cells at a fixed grid spacing. Returning false leaves the launch to
// the next list or to the generic kernel. WDF_GENERIC_ZPASS selects the generic kernel always.
#pragma once

#include <cstdlib>

#include "zpass.cuh"

namespace wdf {

static bool zfast_enabled() {
  static const bool on = std::getenv("WDF_GENERIC_ZPASS") == nullptr;
  return on;
}

template <typename T> static size_t zfast_smem(int n3) { return sizeof(cplx<T>) * (kMaxN + 2 * kZCols * (n3 + 1)); }

template <typename T, int... Ns> struct ZFastSizes {
  template <int N> static bool g2r_n(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {
    if (f.g.n3 != N) return false;
    const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
    launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, false, N>, grid, dim3(kThreads), zfast_smem<T>(N), st, X, nvec, f.g, f.P3, f.tw3,
           cb, PDir<T>());
    WDF_CUDA_TRY(cudaGetLastError());
    return true;
  }
  template <int N> static bool g2r_dir_n(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) {
    if (f.g.n3 != N) return false;
    const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
    launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, true, N>, grid, dim3(kThreads), zfast_smem<T>(N), st, (const cplx<T> *)d.p, nvec,
           f.g, f.P3, f.tw3, cb, d);
    WDF_CUDA_TRY(cudaGetLastError());
    return true;
  }
  template <int N> static bool r2g_n(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
    if (f.g.n3 != N) return false;
    const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
    const size_t sm = zfast_smem<T>(N);
    if (epi == EPI_STORE)
      launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_STORE, N>, grid, dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
    else if (epi == EPI_HSHIFT)
      launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_HSHIFT, N>, grid, dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
    else
      launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI_DRHO, N>, grid, dim3(kThreads), sm, st, cb, nvec, f.g, f.P3, f.tw3, ea);
    WDF_CUDA_TRY(cudaGetLastError());
    return true;
  }
  template <int N> static void limits_n(const Geo &g) {
    if (g.n3 != N) return;
    const size_t sm = zfast_smem<T>(N);
    raise_smem_limit(k_zpass_g2r<T, false, N>, sm);
    raise_smem_limit(k_zpass_g2r<T, true, N>, sm);
    raise_smem_limit(k_zpass_r2g<T, EPI_STORE, N>, sm);
    raise_smem_limit(k_zpass_r2g<T, EPI_HSHIFT, N>, sm);
    raise_smem_limit(k_zpass_r2g<T, EPI_DRHO, N>, sm);
  }
  static bool g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {
    return zfast_enabled() && (g2r_n<Ns>(f, X, nvec, cb, st) || ...);
  }
  static bool g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) {
    return zfast_enabled() && (g2r_dir_n<Ns>(f, d, nvec, cb, st) || ...);
  }
  static bool r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
    return zfast_enabled() && (r2g_n<Ns>(f, epi, cb, nvec, ea, st) || ...);
  }
  static void limits(const Geo &g) { (limits_n<Ns>(g), ...); }
};

// the common sizes (zpass_fast_*.cu) and the further sizes (zpass_more_*.cu)
#define WDF_ZFAST_LIST 24, 30, 32, 40, 48, 64, 80, 96
#define WDF_ZMORE_LIST 36, 45, 50, 54, 60, 72, 75

}  // namespace wdf

// the four entry points for one size list, named PREFIX_g2r and so on (the same definition in
// every translation unit that uses the list), and their instantiation for one precision T
#define WDF_ZFAST_DEFINE(PREFIX, LIST)                                                                                     \
  namespace wdf {                                                                                                         \
  template <typename T> bool PREFIX##_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {  \
    return ZFastSizes<T, LIST>::g2r(f, X, nvec, cb, st);                                                                  \
  }                                                                                                                       \
  template <typename T> bool PREFIX##_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) { \
    return ZFastSizes<T, LIST>::g2r_dir(f, d, nvec, cb, st);                                                              \
  }                                                                                                                       \
  template <typename T>                                                                                                   \
  bool PREFIX##_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {    \
    return ZFastSizes<T, LIST>::r2g(f, epi, cb, nvec, ea, st);                                                            \
  }                                                                                                                       \
  template <typename T> void set_##PREFIX##_limits(const Geo &g) { ZFastSizes<T, LIST>::limits(g); }                     \
  }

#define WDF_ZFAST_INSTANTIATE(T, PREFIX)                                                                                 \
  namespace wdf {                                                                                                         \
  template bool PREFIX##_g2r<T>(const FftCtx<T> &, const cplx<T> *, int, cplx<T> *, cudaStream_t);                      \
  template bool PREFIX##_g2r_dir<T>(const FftCtx<T> &, const PDir<T> &, int, cplx<T> *, cudaStream_t);                 \
  template bool PREFIX##_r2g<T>(const FftCtx<T> &, int, const cplx<T> *, int, const EpiArgs<T> &, cudaStream_t);      \
  template void set_##PREFIX##_limits<T>(const Geo &);                                                                   \
  }

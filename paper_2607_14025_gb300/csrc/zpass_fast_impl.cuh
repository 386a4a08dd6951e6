// Launchers of the compile-time n3 transforms for the grid sizes below (one instantiation per
// size, precision and epilogue; each precision is its own translation unit). Returning false
// leaves the launch to the generic kernel. WDF_GENERIC_ZPASS selects the generic kernel always.
#pragma once

#include <cstdlib>

#include "zpass.cuh"

#define WDF_ZFAST_SIZES(X) X(24) X(30) X(32) X(40) X(48) X(64) X(80) X(96)

namespace wdf {

static bool zfast_enabled() {
  static const bool on = std::getenv("WDF_GENERIC_ZPASS") == nullptr;
  return on;
}

template <typename T> static size_t zfast_smem(int n3) { return sizeof(cplx<T>) * (kMaxN + 2 * kZCols * (n3 + 1)); }

template <typename T> bool zpass_fast_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (!zfast_enabled()) return false;
  const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  switch (f.g.n3) {
#define X(N)                                                                                                                      \
  case N:                                                                                                                         \
    launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, false, N>, grid, dim3(kThreads), zfast_smem<T>(N), st, X, nvec, f.g, f.P3, \
           f.tw3, cb, PDir<T>());                                                                                                  \
    WDF_CUDA_TRY(cudaGetLastError());                                                                                            \
    return true;
    WDF_ZFAST_SIZES(X)
#undef X
    default: return false;
  }
}

template <typename T> bool zpass_fast_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st) {
  if (!zfast_enabled()) return false;
  const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  switch (f.g.n3) {
#define X(N)                                                                                                                  \
  case N:                                                                                                                     \
    launch("zpass_g2r", bits_of<T>(), k_zpass_g2r<T, true, N>, grid, dim3(kThreads), zfast_smem<T>(N), st, (const cplx<T> *)d.p, \
           nvec, f.g, f.P3, f.tw3, cb, d);                                                                                    \
    WDF_CUDA_TRY(cudaGetLastError());                                                                                        \
    return true;
    WDF_ZFAST_SIZES(X)
#undef X
    default: return false;
  }
}

template <typename T, int EPI, int N>
static void zfast_r2g_n(const FftCtx<T> &f, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
  const dim3 grid((nvec + 1) / 2, (f.g.K + kZCols - 1) / kZCols);
  launch("zpass_r2g", bits_of<T>(), k_zpass_r2g<T, EPI, N>, grid, dim3(kThreads), zfast_smem<T>(N), st, cb, nvec, f.g, f.P3, f.tw3, ea);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
bool zpass_fast_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st) {
  if (!zfast_enabled()) return false;
  switch (f.g.n3) {
#define X(N)                                                                       \
  case N:                                                                          \
    if (epi == EPI_STORE) zfast_r2g_n<T, EPI_STORE, N>(f, cb, nvec, ea, st);       \
    else if (epi == EPI_HSHIFT) zfast_r2g_n<T, EPI_HSHIFT, N>(f, cb, nvec, ea, st); \
    else zfast_r2g_n<T, EPI_DRHO, N>(f, cb, nvec, ea, st);                         \
    return true;
    WDF_ZFAST_SIZES(X)
#undef X
    default: return false;
  }
}

template <typename T> void set_zpass_fast_limits(const Geo &g) {
  switch (g.n3) {
#define X(N)                                                            \
  case N: {                                                             \
    const size_t sm = zfast_smem<T>(N);                                 \
    raise_smem_limit(k_zpass_g2r<T, false, N>, sm);                     \
    raise_smem_limit(k_zpass_g2r<T, true, N>, sm);                      \
    raise_smem_limit(k_zpass_r2g<T, EPI_STORE, N>, sm);                 \
    raise_smem_limit(k_zpass_r2g<T, EPI_HSHIFT, N>, sm);                \
    raise_smem_limit(k_zpass_r2g<T, EPI_DRHO, N>, sm);                  \
    break;                                                              \
  }
    WDF_ZFAST_SIZES(X)
#undef X
    default: break;
  }
}

}  // namespace wdf

#define WDF_ZFAST_INST(T)                                                                                             \
  namespace wdf {                                                                                                     \
  template bool zpass_fast_g2r<T>(const FftCtx<T> &, const cplx<T> *, int, cplx<T> *, cudaStream_t);                  \
  template bool zpass_fast_g2r_dir<T>(const FftCtx<T> &, const PDir<T> &, int, cplx<T> *, cudaStream_t);             \
  template bool zpass_fast_r2g<T>(const FftCtx<T> &, int, const cplx<T> *, int, const EpiArgs<T> &, cudaStream_t);  \
  template void set_zpass_fast_limits<T>(const Geo &);                                                               \
  }

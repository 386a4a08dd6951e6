// Internal definitions shared by the translation units of libwdf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "df64.cuh"
#include "wdf.h"

namespace wdf {

// ---------------------------------------------------------------------------------------------
// complex numbers as CUDA vector types (interleaved re, im)

template <typename T> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };
struct __align__(16) cdf64 {
  df64 x, y;
};
template <> struct cplx_t<df64> { typedef cdf64 type; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mkc(T a, T b) {
  cplx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// double-float: each part as one two-product sum (df_dot2)
template <> __device__ __forceinline__ cplx<df64> cmul<df64>(cplx<df64> a, cplx<df64> b) {
  return mkc<df64>(df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x));
}
template <> __device__ __forceinline__ cplx<df64> cmulc<df64>(cplx<df64> a, cplx<df64> b) {
  return mkc<df64>(df_dot2(a.x, b.x, a.y, b.y), df_dot2(a.y, b.x, -a.x, b.y));
}
template <typename T> __device__ __forceinline__ cplx<T> cscal(cplx<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mkc<T>(a.x, -a.y); }
// i * s * a
template <typename T> __device__ __forceinline__ cplx<T> cimul(cplx<T> a, T s) { return mkc<T>(-a.y * s, a.x * s); }

// ---------------------------------------------------------------------------------------------
// one-dimensional FFT plan: mixed radix 4, 2, 3, 5, in place, digit-reversed order on the
// spectral side (see fft.cuh)

constexpr int kMaxStages = 8;
constexpr int kMaxN = 128;

struct Plan1D {
  int n;
  int nst;
  int r[kMaxStages];
  int L[kMaxStages + 1];
};

// ---------------------------------------------------------------------------------------------
// device-side description of the plane-wave layout, passed by value to kernels

struct Geo {
  int n1, n2, n3;     // FFT grid
  int pitch;          // smem row pitch of a plane tile (n1 + 1)
  int K;              // rep columns (column (0,0) first)
  int ndisk;          // disk columns = 2K - 1
  int ldcb;           // stride between z slices of a column buffer (>= ndisk)
  int nint;           // stored elements of one internal vector
  int ld;             // allocated elements per internal vector (>= nint, padded)
  int len0;           // elements of column (0,0) (weight 1; all others weight 2)
  int nxact;          // active x positions of the plane tile
  // device tables
  const int *col_off;      // [K+1] element offset of each rep column (col_off[K] = nint)
  const int *col_zlo;      // [K] lowest n3 of each column
  const int *e_col;        // [nint] column of each element
  const int *e_z;          // [nint] n3 of each element
  const int *tile_idx;     // [ndisk] smem index pos2(i2)*pitch + pos1(i1) of each disk column
  const int *xact;         // [nxact] tile x positions (pos1) with data
  const int *xactn;        // [nxact] the same columns in natural order (n1 mod N1)
  int xmax;                // largest |n1| of the sphere
  int ymax;                // largest |n2| of the sphere
  const short *pos3;       // [n3] digit-reversed position along n3
  const double *g2;        // [ld] |G|^2 of each element (0 in padding)
};

// ---------------------------------------------------------------------------------------------
// error plumbing (host)

struct Error {
  int code = WDF_OK;
  std::string msg;
};

void set_error(int code, const std::string &msg);  // thread-local last error of setup
const char *last_global_error();

}  // namespace wdf

#define WDF_CUDA_TRY(call)                                                                  \
  do {                                                                                      \
    cudaError_t e__ = (call);                                                               \
    if (e__ != cudaSuccess) {                                                               \
      throw ::wdf::CudaFailure(e__, #call, __FILE__, __LINE__);                             \
    }                                                                                       \
  } while (0)

namespace wdf {

// ---------------------------------------------------------------------------------------------
// launch accounting: every kernel launch goes through launch(), which counts it and, when the
// calling thread has selected its class for timing, records CUDA events around it on its stream

struct Profiler {
  std::string target;  // kernel class, e.g. "plane_vloc"
  int bits = 0;        // 64, 32, or 0 for classes without a precision
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  long long count = 0;
  long long blocks = 0;  // work units of the timed launches (thread blocks, or (pair, plane) units of persistent kernels)
};
extern thread_local Profiler *t_prof;
extern std::atomic<long long> g_launches;
void prof_record(cudaStream_t st);  // records the next event of t_prof

// precision tag of a kernel instance: 64 (FP64), 32 (FP32), 48 (double-float)
template <typename T> constexpr int bits_of() { return std::is_same<T, df64>::value ? 48 : (int)(8 * sizeof(T)); }

// `units`: the work units the launch processes (thread blocks, except for persistent kernels)
template <typename... KArgs, typename... Args>
inline void launch_units(const char *cls, int bits, long long units, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args &&...args) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const bool timed = t_prof && t_prof->bits == bits && t_prof->target == cls;
  if (timed) prof_record(st);
  k<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
  if (timed) {
    prof_record(st);
    ++t_prof->count;
    t_prof->blocks += units;
  }
}

template <typename... KArgs, typename... Args>
inline void launch(const char *cls, int bits, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args &&...args) {
  launch_units(cls, bits, (long long)grid.x * grid.y * grid.z, k, grid, block, smem, st, std::forward<Args>(args)...);
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device. The
// attribute belongs to the function, not to a context, so contexts of different grids in one
// process only ever raise it (a smaller later setting would break the larger context's launches).
void raise_smem_limit_raw(const void *func, size_t bytes);
template <typename F> inline void raise_smem_limit(F *func, size_t bytes) { raise_smem_limit_raw((const void *)func, bytes); }

struct CudaFailure {
  cudaError_t err;
  const char *what;
  const char *file;
  int line;
  CudaFailure(cudaError_t e, const char *w, const char *f, int l) : err(e), what(w), file(f), line(l) {}
};
struct ApiFailure {
  int code;
  std::string msg;
  ApiFailure(int c, std::string m) : code(c), msg(std::move(m)) {}
};
}  // namespace wdf

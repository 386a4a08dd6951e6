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

constexpr int GT = 32;  // output tile
constexpr int GK = 32;  // element chunk

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_gram(Geo g, const cplx<T> *__restrict__ A, int na, const cplx<T> *__restrict__ B,
                                             int nb, double *__restrict__ out, int ldo, int echunk, size_t split_stride) {
  __shared__ cplx<T> As[GT][GK + 1];
  __shared__ cplx<T> Bs[GT][GK + 1];
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  const int ebeg = blockIdx.z * echunk;
  const int eend = min(g.nint, ebeg + echunk);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  Acc acc[2][2] = {{0, 0}, {0, 0}};
  for (int e0 = ebeg; e0 < eend; e0 += GK) {
    for (int t = threadIdx.x; t < GT * GK; t += 256) {
      const int row = t / GK, col = t % GK, e = e0 + col;
      const bool ok = e < eend;
      const T w = (T)wgt(e, g.len0);
      cplx<T> a = mkc<T>(0, 0), b = mkc<T>(0, 0);
      if (ok && i0 + row < na) a = A[(size_t)(i0 + row) * g.ld + e];
      if (ok && j0 + row < nb) b = B[(size_t)(j0 + row) * g.ld + e];
      As[row][col] = mkc<T>(a.x * w, a.y * w);
      Bs[row][col] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      const cplx<T> a0 = As[ty * 2][k], a1 = As[ty * 2 + 1][k];
      const cplx<T> b0 = Bs[tx * 2][k], b1 = Bs[tx * 2 + 1][k];
      acc[0][0] += (Acc)a0.x * (Acc)b0.x + (Acc)a0.y * (Acc)b0.y;
      acc[0][1] += (Acc)a0.x * (Acc)b1.x + (Acc)a0.y * (Acc)b1.y;
      acc[1][0] += (Acc)a1.x * (Acc)b0.x + (Acc)a1.y * (Acc)b0.y;
      acc[1][1] += (Acc)a1.x * (Acc)b1.x + (Acc)a1.y * (Acc)b1.y;
    }
    __syncthreads();
  }
  double *o = out + blockIdx.z * split_stride;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty * 2 + a, j = j0 + tx * 2 + b;
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

static int gram_nsplit(const Geo &g, int na, int nb, int &echunk) {
  const int tiles = ((na + GT - 1) / GT) * ((nb + GT - 1) / GT);
  int nsplit = 1;
  const int target = 2 * 152;  // two waves of blocks on the 152 SMs
  if (tiles < target) nsplit = std::min(64, std::max(1, target / tiles));
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
  int echunk;
  int nsplit = gram_nsplit(g, na, nb, echunk);
  const size_t stride = (size_t)na * ldo;
  if (nsplit > 1 && (work == nullptr || work_cap < stride * nsplit)) {
    nsplit = 1;
    echunk = ((g.nint + GK - 1) / GK) * GK;
  }
  dim3 grid((na + GT - 1) / GT, (nb + GT - 1) / GT, nsplit);
  typedef typename std::conditional<std::is_same<T, double>::value, double, float>::type Acc;
  if (nsplit == 1) {
    k_gram<T, Acc><<<grid, 256, 0, st>>>(g, A, na, B, nb, out, ldo, echunk, 0);
  } else {
    k_gram<T, Acc><<<grid, 256, 0, st>>>(g, A, na, B, nb, work, ldo, echunk, stride);
    WDF_CUDA_TRY(cudaGetLastError());
    k_sum_splits<<<(na * nb + 255) / 256, 256, 0, st>>>(work, nsplit, stride, out, na, nb, ldo);
  }
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// linear combinations Y_s = c0 Y_s + sum_j U_j C[j][s] d_j

constexpr int LE = 64;  // elements per block
constexpr int LS = 16;  // vectors per block
constexpr int LJ = 32;  // coefficient rows staged at a time

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) k_lincomb(Geo g, cplx<T> *__restrict__ Y, int ny, const cplx<T> *__restrict__ U, int nu,
                                                const double *__restrict__ C, int ldc, const double *__restrict__ d, double c0) {
  __shared__ Acc cs[LJ][LS];
  const int e = blockIdx.x * LE + (threadIdx.x % LE);
  const int sg = threadIdx.x / LE;  // 0..3, four vectors each
  const int s0 = blockIdx.y * LS;
  Acc ax[4] = {0, 0, 0, 0}, ay[4] = {0, 0, 0, 0};
  for (int j0 = 0; j0 < nu; j0 += LJ) {
    for (int t = threadIdx.x; t < LJ * LS; t += 256) {
      const int jj = t / LS, ss = t % LS;
      const int j = j0 + jj, s = s0 + ss;
      double v = 0.0;
      if (j < nu && s < ny) v = C[(size_t)j * ldc + s] * (d ? d[j] : 1.0);
      cs[jj][ss] = (Acc)v;
    }
    __syncthreads();
    if (e < g.nint) {
      const int jn = min(LJ, nu - j0);
      for (int jj = 0; jj < jn; ++jj) {
        const cplx<T> u = U[(size_t)(j0 + jj) * g.ld + e];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const Acc c = cs[jj][sg * 4 + k];
          ax[k] += c * (Acc)u.x;
          ay[k] += c * (Acc)u.y;
        }
      }
    }
    __syncthreads();
  }
  if (e >= g.nint) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int s = s0 + sg * 4 + k;
    if (s >= ny) continue;
    cplx<T> *y = Y + (size_t)s * g.ld + e;
    if (c0 == 0.0) {
      *y = mkc<T>((T)ax[k], (T)ay[k]);
    } else {
      const cplx<T> o = *y;
      *y = mkc<T>((T)((Acc)c0 * (Acc)o.x + ax[k]), (T)((Acc)c0 * (Acc)o.y + ay[k]));
    }
  }
}

template <typename T>
void launch_lincomb(const Geo &g, cplx<T> *Y, int ny, const cplx<T> *U, int nu, const double *C, int ldc, const double *d,
                    double c0, cudaStream_t st) {
  if (ny <= 0) return;
  dim3 grid((g.nint + LE - 1) / LE, (ny + LS - 1) / LS);
  typedef typename std::conditional<std::is_same<T, double>::value, double, float>::type Acc;
  k_lincomb<T, Acc><<<grid, 256, 0, st>>>(g, Y, ny, U, nu, C, ldc, d, c0);
  WDF_CUDA_TRY(cudaGetLastError());
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
  k_dot_partial<T><<<dim3(nvec, nchunk), 256, 0, st>>>(g, A, B, part, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// conjugate gradients

template <typename T>
__global__ void __launch_bounds__(256) k_cg_start(Geo g, const cplx<T> *__restrict__ r, cplx<T> *__restrict__ z,
                                                 cplx<T> *__restrict__ p, const T *__restrict__ kprec, CgState s, int nchunk) {
  const int i = blockIdx.x, c = blockIdx.y;
  const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
  const size_t o = (size_t)i * g.ld;
  const T *K = kprec ? kprec + (size_t)s.vidx[i] * g.ld : nullptr;
  double vrz = 0.0, vrr = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const cplx<T> rv = r[o + e];
    const T k = K ? K[e] : (T)1;
    const cplx<T> zv = mkc<T>(k * rv.x, k * rv.y);
    z[o + e] = zv;
    p[o + e] = zv;
    const double w = wgt(e, g.len0);
    vrz += w * dre<T>(rv, zv);
    vrr += w * dre<T>(rv, rv);
  }
  vrz = block_sum(vrz);
  vrr = block_sum(vrr);
  if (threadIdx.x == 0) {
    s.part1[(size_t)i * nchunk + c] = vrz;
    s.part2[(size_t)i * nchunk + c] = vrr;
  }
}

template <typename T>
void launch_cg_start(const Geo &g, const cplx<T> *r, cplx<T> *z, cplx<T> *p, const T *kprec, const CgState &s, int n, int nchunk,
                     cudaStream_t st) {
  if (n <= 0) return;
  k_cg_start<T><<<dim3(n, nchunk), 256, 0, st>>>(g, r, z, p, kprec, s, nchunk);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(Geo g, cplx<T> *__restrict__ x, cplx<T> *__restrict__ r, cplx<T> *__restrict__ z,
                                                  const cplx<T> *__restrict__ p, const cplx<T> *__restrict__ Ap,
                                                  const T *__restrict__ kprec, CgState s, int nchunk) {
  const int i = blockIdx.x, c = blockIdx.y;
  double vrz = 0.0, vrr = 0.0;
  if (s.active[i]) {
    const int e0 = c * DCHUNK, e1 = min(g.nint, e0 + DCHUNK);
    const size_t o = (size_t)i * g.ld;
    const T *K = kprec ? kprec + (size_t)s.vidx[i] * g.ld : nullptr;
    const T al = (T)(s.rz[i] / s.pap[i]);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const cplx<T> pv = p[o + e], av = Ap[o + e];
      cplx<T> xv = x[o + e], rv = r[o + e];
      xv.x += al * pv.x;
      xv.y += al * pv.y;
      rv.x -= al * av.x;
      rv.y -= al * av.y;
      x[o + e] = xv;
      r[o + e] = rv;
      const T k = K ? K[e] : (T)1;
      const cplx<T> zv = mkc<T>(k * rv.x, k * rv.y);
      z[o + e] = zv;
      const double w = wgt(e, g.len0);
      vrz += w * dre<T>(rv, zv);
      vrr += w * dre<T>(rv, rv);
    }
  }
  vrz = block_sum(vrz);
  vrr = block_sum(vrr);
  if (threadIdx.x == 0) {
    s.part1[(size_t)i * nchunk + c] = vrz;
    s.part2[(size_t)i * nchunk + c] = vrr;
  }
}

template <typename T>
void launch_cg_update(const Geo &g, cplx<T> *x, cplx<T> *r, cplx<T> *z, const cplx<T> *p, const cplx<T> *Ap, const T *kprec,
                      const CgState &s, int n, int nchunk, cudaStream_t st) {
  if (n <= 0) return;
  k_cg_update<T><<<dim3(n, nchunk), 256, 0, st>>>(g, x, r, z, p, Ap, kprec, s, nchunk);
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
  k_cg_direction<T><<<dim3(n, by), 256, 0, st>>>(g, p, z, s, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

__global__ void k_cg_scalars(CgState s, int n, int nchunk, int which, int maxiter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0, b = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    a += s.part1[(size_t)i * nchunk + c];
    b += s.part2[(size_t)i * nchunk + c];
  }
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
  } else {
    atomicAdd(s.nactive, 1);
  }
}

void launch_cg_scalars(const CgState &s, int n, int nchunk, int which, int maxiter, cudaStream_t st) {
  if (n <= 0) return;
  k_cg_scalars<<<(n + 127) / 128, 128, 0, st>>>(s, n, nchunk, which, maxiter);
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
  k_axpby<T><<<std::min(4096, (int)(((size_t)n * g.ld + 255) / 256)), 256, 0, st>>>(g, y, x, n, a, b);
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
  k_scale_rows<T><<<std::min(4096, (int)(((size_t)n * g.ld + 255) / 256)), 256, 0, st>>>(g, y, coef, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename Tin, typename Tout>
__global__ void k_convert(Tout *__restrict__ y, const Tin *__restrict__ x, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) y[t] = (Tout)x[t];
}
template <typename Tin, typename Tout> void launch_convert(const Geo &, Tout *y, const Tin *x, size_t count, cudaStream_t st) {
  if (count == 0) return;
  k_convert<Tin, Tout><<<(int)std::min<size_t>(8192, (count + 255) / 256), 256, 0, st>>>(y, x, count);
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
  k_ext_to_int<<<(int)std::min<size_t>(8192, (tot + 255) / 256), 256, 0, st>>>(ext, n, npw_h, emap, emap2, econj, scale_int, out, ld);
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
  k_int_to_ext<<<(int)std::min<size_t>(8192, (tot + 255) / 256), 256, 0, st>>>(in, n, ld, npw_h, emap, econj, ext);
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
  k_ritz_residual<<<std::min(4096, (int)(((size_t)n * g.ld + 255) / 256)), 256, 0, st>>>(g, R, AX, X, theta, n);
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
  k_tpa_table<T><<<std::min(4096, (int)(((size_t)n * g.ld + 255) / 256)), 256, 0, st>>>(g, K, tkin, n);
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
  k_kinetic<<<n, 256, 0, st>>>(g, X, tkin);
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
  k_mul_table<T><<<std::min(4096, (int)(((size_t)n * g.ld + 255) / 256)), 256, 0, st>>>(g, y, tab, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void k_check_finite(const T *__restrict__ x, size_t count, int *flag) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[t])) atomicExch(flag, 1);
}
template <typename T> void launch_check_finite(const T *x, size_t count, int *flag, cudaStream_t st) {
  if (count == 0) return;
  k_check_finite<T><<<(int)std::min<size_t>(4096, (count + 255) / 256), 256, 0, st>>>(x, count, flag);
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

size_t jacobi_work_doubles(int n) {
  const int m = std::max(2, n + (n & 1));
  return 2 * (size_t)m * m + 2 * (size_t)m;
}

void jacobi_eigh(double *Ain, double *Vout, double *w, int n, double *work, int *iwork, cudaStream_t st) {
  if (n <= 0) return;
  const int mm = std::max(2, n + (n & 1));
  double *A = work, *V = work + (size_t)mm * mm, *cs = V + (size_t)mm * mm;
  int *done = iwork;
  k_jac_init<<<std::min(1024, (mm * mm + 255) / 256), 256, 0, st>>>(Ain, n, A, V, mm, done);
  WDF_CUDA_TRY(cudaGetLastError());
  const int maxsweep = 40;
  int hdone = 0;
  for (int sweep = 0; sweep < maxsweep && !hdone; ++sweep) {
    for (int rd = 0; rd < mm - 1; ++rd) {
      k_jac_rows<<<mm / 2, 128, 0, st>>>(A, mm, rd, cs, done);
      k_jac_cols<<<mm / 2, 128, 0, st>>>(A, V, mm, rd, cs, done);
    }
    k_jac_check<<<1, 1024, 0, st>>>(A, mm, done);
    WDF_CUDA_TRY(cudaGetLastError());
    if (sweep % 3 == 2) {
      WDF_CUDA_TRY(cudaMemcpyAsync(&hdone, done, sizeof(int), cudaMemcpyDeviceToHost, st));
      WDF_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  k_jac_sort<<<1, 256, 0, st>>>(A, V, mm, n, w, Vout);
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

}  // namespace wdf

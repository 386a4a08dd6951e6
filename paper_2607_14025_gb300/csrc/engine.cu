// Solver engine: Hamiltonian and Sternheimer operators, preconditioned CG with iterative
// refinement, chi0bar application by DFPT and the block Davidson shared by the ground state and
// PDEP (paper Sec. 2.1 for the method, Sec. 3.3 for the single Davidson implementation).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "engine.cuh"

namespace wdf {

// ---------------------------------------------------------------------------------------------
// small local kernels

template <typename T>
__global__ void k_split_pairs(const cplx<T> *__restrict__ grid, int npair, size_t ngrid, T *__restrict__ out, int nreal) {
  const size_t tot = (size_t)npair * ngrid;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / ngrid);
    const size_t i = t % ngrid;
    const cplx<T> v = grid[t];
    out[(size_t)(2 * q) * ngrid + i] = v.x;
    if (2 * q + 1 < nreal) out[(size_t)(2 * q + 1) * ngrid + i] = v.y;
  }
}

__global__ void k_scale_elems(Geo g, cplx<double> *__restrict__ y, const cplx<double> *__restrict__ x, const double *__restrict__ tab,
                              int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x)
    y[t] = cscal<double>(x[t], tab[t % g.ld]);
}

__global__ void k_gather_shift(const int *__restrict__ vidx, const double *__restrict__ eps, double *__restrict__ shift, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) shift[t] = eps[vidx[t]];
}

__global__ void k_sum_chunks(const double *__restrict__ part, int n, int nchunk, double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)t * nchunk + c];
  out[t] = s;
}

static int grid_for(size_t tot) { return (int)std::min<size_t>(8192, (tot + 255) / 256); }

// ---------------------------------------------------------------------------------------------
// compaction of the active solves of a CG batch

// per-solve state that moves with the rows (krow: preconditioner row; home: row of the caller's x,
// -1 for a padding row; rr_ref, it_ref, vorig: learned preconditioner only, may be null)
struct CgRows {
  double *rz, *rz_new, *thr, *shift, *rr_ref;
  int *active, *iters, *krow, *vorig, *it_ref, *home;
};

// src[k] = the k-th active row, in increasing order (one block of 1024 threads, chunked scan)
__global__ void __launch_bounds__(1024) k_compact_index(const int *__restrict__ active, int n, int *__restrict__ src) {
  __shared__ int sums[1024];
  const int t = threadIdx.x, per = (n + 1023) / 1024;
  const int b = min(n, t * per), e = min(n, b + per);
  int c = 0;
  for (int i = b; i < e; ++i) c += active[i] ? 1 : 0;
  sums[t] = c;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int pos = sums[t] - c;
  for (int i = b; i < e; ++i)
    if (active[i]) src[pos++] = i;
}

__global__ void k_compact_scalars(CgRows a, CgRows b, const int *__restrict__ src, int nnew, int nact) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnew) return;
  if (k < nact) {
    const int i = src[k];
    b.rz[k] = a.rz[i];
    b.rz_new[k] = a.rz_new[i];
    b.thr[k] = a.thr[i];
    b.shift[k] = a.shift[i];
    if (b.rr_ref) b.rr_ref[k] = a.rr_ref[i];
    b.active[k] = a.active[i];
    b.iters[k] = a.iters[i];
    b.krow[k] = a.krow[i];
    if (b.vorig) b.vorig[k] = a.vorig[i];
    if (b.it_ref) b.it_ref[k] = a.it_ref[i];
    b.home[k] = a.home ? a.home[i] : i;
  } else {  // padding row that completes the last pair: inactive, zero vectors
    b.rz[k] = 1.0;
    b.rz_new[k] = 0.0;
    b.thr[k] = 1e300;
    b.shift[k] = 0.0;
    if (b.rr_ref) b.rr_ref[k] = 0.0;
    b.active[k] = 0;
    b.iters[k] = 0;
    b.krow[k] = a.krow[0];
    if (b.vorig) b.vorig[k] = 0;
    if (b.it_ref) b.it_ref[k] = 0;
    b.home[k] = -1;
  }
}

template <typename T>
__global__ void k_compact_vectors(Geo g, const cplx<T> *__restrict__ r, const cplx<T> *__restrict__ p, cplx<T> *__restrict__ r2,
                                  cplx<T> *__restrict__ p2, const int *__restrict__ src, int nnew, int nact) {
  const size_t tot = (size_t)nnew * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / g.ld), e = (int)(t % g.ld);
    if (k < nact) {
      const size_t o = (size_t)src[k] * g.ld + e;
      r2[t] = r[o];
      p2[t] = p[o];
    } else {
      r2[t] = mkc<T>(0, 0);
      p2[t] = mkc<T>(0, 0);
    }
  }
}

// iteration counts (and preconditioner rows) of the current rows back to the caller's order
__global__ void k_scatter_home(CgRows a, int n, int *__restrict__ iters_home, int *__restrict__ krow_home) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int h = a.home ? a.home[k] : k;
  if (h < 0) return;
  iters_home[h] = a.iters[k];
  if (krow_home) krow_home[h] = a.krow[k];
}

// ---------------------------------------------------------------------------------------------
// precision traits

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const FftCtx<double> &f(wdf_ctx *c) { return c->f64; }
  static const double *vloc(wdf_ctx *c) { return c->vloc64.as<double>(); }
  static const cplx<double> *U(wdf_ctx *c) { return c->U64.as<cplx<double>>(); }
  static const double *kp(wdf_ctx *c) { return c->kp64.as<double>(); }
  static const double *ml(wdf_ctx *c) { return c->ml64.as<double>(); }
  static wdf_ctx::Cg &cg(wdf_ctx *c) { return c->cg64; }
};
template <> struct Prec<float> {
  static const FftCtx<float> &f(wdf_ctx *c) { return c->f32; }
  static const float *vloc(wdf_ctx *c) { return c->vloc32.as<float>(); }
  static const cplx<float> *U(wdf_ctx *c) { return c->U32.as<cplx<float>>(); }
  static const float *kp(wdf_ctx *c) { return c->kp32.as<float>(); }
  static const float *ml(wdf_ctx *c) { return c->ml32.as<float>(); }
  static wdf_ctx::Cg &cg(wdf_ctx *c) { return c->cg32; }
};
template <> struct Prec<df64> {
  static const FftCtx<df64> &f(wdf_ctx *c) { return c->fdf; }
  static const df64 *vloc(wdf_ctx *c) { return c->vlocdf.as<df64>(); }
  static const cplx<df64> *U(wdf_ctx *c) { return c->Udf.as<cplx<df64>>(); }
  static wdf_ctx::Cg &cg(wdf_ctx *c) { return c->cgdf; }
};

// buffers of the right-hand-side / density-response stage in FP64 or double-float
template <typename R> struct Stage;
template <> struct Stage<double> {
  static const double *psir(wdf_ctx *c) { return c->psir64.as<double>(); }
  static DBuf &dv(wdf_ctx *c) { return c->dvgrid; }
  static DBuf &acc(wdf_ctx *c) { return c->accgrid; }
  static DBuf &cb2(wdf_ctx *c) { return c->cb2; }
  static DBuf &fields(wdf_ctx *c) { return c->orbfields; }
  static DBuf &ones(wdf_ctx *c) { return c->ones64; }
};
template <> struct Stage<df64> {
  static const df64 *psir(wdf_ctx *c) { return c->psirdf.as<df64>(); }
  static DBuf &dv(wdf_ctx *c) { return c->dvgriddf; }
  static DBuf &acc(wdf_ctx *c) { return c->accgriddf; }
  static DBuf &cb2(wdf_ctx *c) { return c->cb2df; }
  static DBuf &fields(wdf_ctx *c) { return c->orbfields; }
  static DBuf &ones(wdf_ctx *c) { return c->onesdf; }
};

// FP64 complex vectors <-> double-float complex vectors (n rows of ld)
static void to_df(wdf_ctx *c, cplx<df64> *y, const cplx<double> *x, size_t nrows) {
  launch_convert<double, df64>(c->geo, (df64 *)y, (const double *)x, 2 * nrows * c->geo.ld, c->st);
}
static void from_df(wdf_ctx *c, cplx<double> *y, const cplx<df64> *x, size_t nrows) {
  launch_convert<df64, double>(c->geo, (double *)y, (const df64 *)x, 2 * nrows * c->geo.ld, c->st);
}

static const double *zeros(wdf_ctx *c, size_t n) {
  if (c->zeros.cap < n * sizeof(double)) {
    c->zeros.ensure(n * sizeof(double));
    WDF_CUDA_TRY(cudaMemsetAsync(c->zeros.p, 0, c->zeros.cap, c->st));
  }
  return c->zeros.as<double>();
}

static double *gram_work(wdf_ctx *c, int na, int nb, int ldo, size_t &cap) {
  const size_t need = gram_work_doubles(c->geo, na, nb, ldo);
  c->gramw.ensure(std::max<size_t>(need, 1) * sizeof(double));
  cap = c->gramw.cap / sizeof(double);
  return c->gramw.as<double>();
}

template <typename T>
static void gram(wdf_ctx *c, const cplx<T> *A, int na, const cplx<T> *B, int nb, double *out, int ldo) {
  size_t cap;
  double *w = gram_work(c, na, nb, ldo, cap);
  launch_gram<T>(c->geo, A, na, B, nb, out, ldo, w, cap, c->st);
}

// digit matrix of rows x K values in (dig, ex), grown on demand
static OzMat oz_mat(DBuf &dig, DBuf &ex, int rows, int K) {
  OzMat m;
  m.rows = rows;
  m.kpad = oz_kpad(K);
  m.plane = (size_t)rows * m.kpad;
  dig.ensure(sizeof(uint16_t) * OZ_DIGITS * std::max<size_t>(m.plane, 1));
  ex.ensure(sizeof(int) * std::max(rows, 1));
  m.dig = dig.as<uint16_t>();
  m.ex = ex.as<int>();
  return m;
}

// Low-rank part on the tensor cores in double-float: Y = c0 Y + Bt (d o (A^T X)) with A the
// weighted rows j0 .. j0 + na - 1 of U (digits c->oz_u) and Bt the matching digits of U^T (all
// rows of U, or the orbital rows). S (na x n doubles, row stride n) receives the projections.
static void oz_lowrank(wdf_ctx *c, int j0, int na, const OzMat &Bt, const cplx<df64> *X, cplx<df64> *Y, int n, const double *d, float c0,
                       double *S) {
  const Geo &g = c->geo;
  const int kf = 2 * g.nint;
  const OzMat A = c->oz_u.sub(j0, na);
  // the vectors' digits in chunks of at most 8,192 rows (5.3 GB of digits at 96^3)
  const int chunk = std::min(n, 8192);
  for (int s0 = 0; s0 < n; s0 += chunk) {
    const int ns = std::min(chunk, n - s0);
    const OzMat Xd = oz_mat(c->ozX, c->ozXe, ns, kf);
    launch_oz_rows_df(g, X + (size_t)s0 * g.ld, ns, false, Xd, c->st);
    const size_t need = oz_gram_work_doubles(na, ns, kf);
    c->gramw.ensure(sizeof(double) * std::max<size_t>(need, 1));
    launch_oz_gram(A, Xd, kf, S + s0, n, c->gramw.as<double>(), c->gramw.cap / sizeof(double), c->tcerr.as<int>(), c->st);
  }
  const OzMat Cd = oz_mat(c->ozC, c->ozCe, n, na);
  launch_oz_cols(S, (size_t)n, na, n, d, Cd, c->st);
  OzMat B = Bt;
  launch_oz_lincomb(Cd, B, na, reinterpret_cast<df64 *>(Y), (size_t)2 * g.ld, c0, c->tcerr.as<int>(), c->st);
}

// per-vector inner products <A_s, B_s> into a device array (n doubles)
template <typename T>
static void dots(wdf_ctx *c, const cplx<T> *A, const cplx<T> *B, int n, double *out) {
  const int nch = dot_chunks(c->geo);
  wdf_ctx::Cg &w = Prec<T>::cg(c);
  w.part1.ensure(sizeof(double) * (size_t)n * nch);
  launch_dot_partial<T>(c->geo, A, B, n, w.part1.as<double>(), nch, c->st);
  launch("sum_chunks", 0, k_sum_chunks, dim3((n + 127) / 128), dim3(128), 0, c->st, w.part1.as<double>(), n, nch, out);
  WDF_CUDA_TRY(cudaGetLastError());
}

static std::vector<double> to_host(wdf_ctx *c, const double *d, size_t n) {
  std::vector<double> h(n);
  if (n) {
    WDF_CUDA_TRY(cudaMemcpyAsync(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  return h;
}

// ---------------------------------------------------------------------------------------------
// operators

// Pairs of solves per pass of the three FFT kernels (n3 inverse, plane, n3 forward) of an operator
// application. With a budget of B MB the column buffer of one pass (n3 ldcb complex values per
// pair) stays within B MB, so the plane kernel and the forward n3 transforms could read what the
// inverse ones wrote from L2 (129 MB) instead of HBM. Measured on the 64^3 system (8,192 solves):
// 443 ms per step in one pass, 458 / 465 / 481 ms with 96 / 64 / 32 MB passes; the extra launches
// and the shorter loops of the persistent plane kernel cost more than the L2 residency saves, so
// the default is one pass. WDF_FFT_CHUNK_MB sets the budget (0 or unset: one pass).
static int fft_chunk_pairs(const Geo &g, size_t elem_bytes, int npair) {
  static const long budget_mb = [] {
    const char *e = std::getenv("WDF_FFT_CHUNK_MB");
    return e ? std::atol(e) : 0L;
  }();
  if (budget_mb <= 0 || npair <= 1) return std::max(1, npair);
  const size_t per_pair = elem_bytes * (size_t)g.n3 * g.ldcb;
  const int cp = (int)std::max<size_t>(1, ((size_t)budget_mb << 20) / per_pair);
  if (cp >= npair) return npair;
  const int nchunk = (npair + cp - 1) / cp;
  return (npair + nchunk - 1) / nchunk;  // even chunks
}

// Y = (H - shift_s) X (+ alpha P X when with_alpha); H = 1/2|G|^2 + V_loc + sum_j beta_j D_j beta_j^T
template <typename T>
void apply_operator(wdf_ctx *c, const cplx<T> *X, cplx<T> *Y, int n, const double *shift, bool with_alpha) {
  if (n <= 0) return;
  const FftCtx<T> &f = Prec<T>::f(c);
  const Geo &g = c->geo;
  wdf_ctx::Cg &w = Prec<T>::cg(c);
  const int npair = (n + 1) / 2;
  const int cp = fft_chunk_pairs(g, sizeof(cplx<T>), npair);
  w.cb.ensure(sizeof(cplx<T>) * (size_t)cp * g.n3 * g.ldcb);
  cplx<T> *cb = w.cb.as<cplx<T>>();
  const double *sh = shift ? shift : zeros(c, n);
  for (int p0 = 0; p0 < npair; p0 += cp) {
    const int s0 = 2 * p0, ns = std::min(n - s0, 2 * cp), np = (ns + 1) / 2;
    launch_zpass_g2r<T>(f, X + (size_t)s0 * g.ld, ns, cb, c->st);
    PlaneArgs<T> pa;
    pa.cb = cb;
    pa.field = Prec<T>::vloc(c);
    launch_plane<T>(f, OP_VLOC, np, pa, c->st);
    EpiArgs<T> ea;
    ea.Y = Y + (size_t)s0 * g.ld;
    ea.X = X + (size_t)s0 * g.ld;
    ea.shift = sh + s0;
    ea.scale = (T)(1.0 / (double)c->ngrid);
    launch_zpass_r2g<T>(f, EPI_HSHIFT, cb, ns, ea, c->st);
  }
  const int M = c->nproj + (with_alpha ? c->nocc : 0);
  if constexpr (std::is_same<T, df64>::value) {
    if (M > 0 && c->oz_on) {
      w.S.ensure(sizeof(double) * (size_t)M * n);
      oz_lowrank(c, 0, M, c->oz_ut, X, Y, n, c->lrd.as<double>(), 1.f, w.S.as<double>());
      return;
    }
  }
  if (M > 0) {
    w.S.ensure(sizeof(double) * (size_t)M * n);
    gram<T>(c, Prec<T>::U(c), M, X, n, w.S.as<double>(), n);
    launch_lincomb<T>(g, Y, n, Prec<T>::U(c), M, w.S.as<double>(), n, c->lrd.as<double>(), 1.0, c->st);
  }
}

// The CG's operator application: like apply_operator with the shift and the occupied-space term,
// plus (dir != null) the direction update p = K r + beta p folded into the first transform, and
// the partial sums of <p, A p> from the epilogue of the last linear combination. Returns the
// number of partial sums per solve written to dotpart, or 0 if they were not computed.
template <typename T>
static int apply_operator_cg(wdf_ctx *c, cplx<T> *X, cplx<T> *Y, int n, const double *shift, const PDir<T> *dir, double *dotpart) {
  const FftCtx<T> &f = Prec<T>::f(c);
  const Geo &g = c->geo;
  wdf_ctx::Cg &w = Prec<T>::cg(c);
  const int npair = (n + 1) / 2;
  const int cp = fft_chunk_pairs(g, sizeof(cplx<T>), npair);
  w.cb.ensure(sizeof(cplx<T>) * (size_t)cp * g.n3 * g.ldcb);
  cplx<T> *cb = w.cb.as<cplx<T>>();
  for (int p0 = 0; p0 < npair; p0 += cp) {  // chunks of pairs whose column buffer stays in L2
    const int s0 = 2 * p0, ns = std::min(n - s0, 2 * cp), np = (ns + 1) / 2;
    const size_t off = (size_t)s0 * g.ld;
    if (dir) {
      PDir<T> d = *dir;
      d.p += off;
      d.r += off;
      d.vidx += s0;
      d.active += s0;
      d.beta += s0;
      launch_zpass_g2r_dir<T>(f, d, ns, cb, c->st);
    } else {
      launch_zpass_g2r<T>(f, X + off, ns, cb, c->st);
    }
    PlaneArgs<T> pa;
    pa.cb = cb;
    pa.field = Prec<T>::vloc(c);
    launch_plane<T>(f, OP_VLOC, np, pa, c->st);
    EpiArgs<T> ea;
    ea.Y = Y + off;
    ea.X = X + off;
    ea.shift = shift + s0;
    ea.scale = (T)(1.0 / (double)c->ngrid);
    launch_zpass_r2g<T>(f, EPI_HSHIFT, cb, ns, ea, c->st);
  }
  const int M = c->nproj + c->nocc;
  w.S.ensure(sizeof(double) * (size_t)M * n);
  if constexpr (std::is_same<T, float>::value) {
    if (c->tc_on) {  // tensor-core (3xTF32) projections
      size_t cap = 0;
      const size_t need = gram_tc_work_doubles(g, M, n);
      c->gramw.ensure(std::max<size_t>(need, 1) * sizeof(double));
      cap = c->gramw.cap / sizeof(double);
      launch_gram_tc(g, reinterpret_cast<const float *>(X), n, c->tc_uwh(), c->tc_uwl(), M, w.S.as<double>(), c->gramw.as<double>(),
                     cap, c->tcerr.as<int>(), c->st);
      const int kp = tc_rows(M);
      c->tcC.ensure(sizeof(float) * 2 * (size_t)n * kp);
      float *chi = c->tcC.as<float>(), *clo = chi + (size_t)n * kp;
      launch_lincomb_tc(g, reinterpret_cast<float *>(Y), n, w.S.as<double>(), n, c->lrd.as<double>(), M, chi, clo, c->tc_uth(),
                        c->tc_utl(), 1.0f, dotpart ? reinterpret_cast<const float *>(X) : nullptr, dotpart, c->tcerr.as<int>(), c->st);
      return dotpart ? lincomb_dot_chunks(g) : 0;
    }
  }
  gram<T>(c, Prec<T>::U(c), M, X, n, w.S.as<double>(), n);
  if (launch_lincomb_dot<T>(g, Y, n, Prec<T>::U(c), M, w.S.as<double>(), n, c->lrd.as<double>(), 1.0, X, dotpart, c->st))
    return lincomb_dot_chunks(g);
  launch_lincomb<T>(g, Y, n, Prec<T>::U(c), M, w.S.as<double>(), n, c->lrd.as<double>(), 1.0, c->st);
  return 0;
}

// ---------------------------------------------------------------------------------------------
// preconditioned conjugate gradients on (H - eps_v + alpha P) d = b, one solve per row

template <typename T>
static void cg_solve(wdf_ctx *c, const cplx<T> *b, cplx<T> *x, int n, int maxiter, std::vector<int> &iters) {
  const Geo &g = c->geo;
  wdf_ctx::Cg &w = Prec<T>::cg(c);
  const size_t vb = sizeof(cplx<T>) * (size_t)n * g.ld;
  w.r.ensure(vb);
  w.z.ensure(vb);
  w.p.ensure(vb);
  w.Ap.ensure(vb);
  const int nch = dot_chunks(g);
  w.part1.ensure(sizeof(double) * (size_t)n * std::max(nch, lincomb_dot_chunks(g)));
  w.part2.ensure(sizeof(double) * (size_t)n * nch);
  w.dbl.ensure(sizeof(double) * 4 * (size_t)n);
  w.ints.ensure(sizeof(int) * (2 * (size_t)n + 1));
  CgState s;
  double *d = w.dbl.as<double>();
  s.rz = d;
  s.rz_new = d + n;
  s.pap = d + 2 * n;
  s.rr = d + 3 * n;
  s.thr = c->thr.as<double>();
  s.shift = c->shift.as<double>();
  s.part1 = w.part1.as<double>();
  s.part2 = w.part2.as<double>();
  int *ii = w.ints.as<int>();
  s.active = ii;
  s.iters = ii + n;
  s.nactive = ii + 2 * n;
  s.vidx = c->vidx_dev.as<int>();
  cplx<T> *r = w.r.as<cplx<T>>(), *z = w.z.as<cplx<T>>(), *p = w.p.as<cplx<T>>(), *Ap = w.Ap.as<cplx<T>>();
  cudaStream_t st = c->st;
  const T *K = c->opt.precond == WDF_PRECOND_TPA ? Prec<T>::kp(c) : nullptr;
  if (c->opt.precond == WDF_PRECOND_LEARNED) {
    // rows of the [learned; TPA] table per solve; the row index moves to TPA on a stall
    K = Prec<T>::ml(c);
    w.part3.ensure(sizeof(double) * (size_t)n * nch);
    s.krow = c->krow.as<int>();
    s.vidx = s.krow;
    s.vorig = c->vidx_dev.as<int>();
    s.nocc = c->nocc;
    s.rr_ref = c->rr_ref.as<double>();
    s.it_ref = c->it_ref.as<int>();
    s.part3 = w.part3.as<double>();
    s.nfb = c->nfb.as<int>();
  }

  WDF_CUDA_TRY(cudaMemsetAsync(x, 0, vb, st));
  WDF_CUDA_TRY(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, st));
  WDF_CUDA_TRY(cudaMemsetAsync(ii, 0, sizeof(int) * (2 * (size_t)n + 1), st));
  (void)z;  // z = K r is not stored: the update and the direction recompute it
  launch_cg_start<T>(g, r, nullptr, p, K, s, n, nch, st);
  launch_cg_scalars(s, n, nch, 2, maxiter, st);
  int nact = 0;
  WDF_CUDA_TRY(cudaMemcpyAsync(&nact, s.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
  WDF_CUDA_TRY(cudaStreamSynchronize(st));
  // Rows of the batch: the home set (the caller's order) and two compacted sets. When enough
  // solves have converged, the active ones are gathered into a dense prefix (r, p and the
  // per-solve state; x stays in the caller's order and is reached through home[]), so the FFTs
  // and projections of later iterations only touch solves that still iterate.
  const bool learned = s.krow != nullptr;
  static const bool compaction = std::getenv("WDF_NO_COMPACT") == nullptr;
  CgRows cur{s.rz, s.rz_new, s.thr, s.shift, s.rr_ref, s.active, s.iters, s.vidx, const_cast<int *>(s.vorig), s.it_ref, nullptr};
  int ncur = n, nset = 0;
  w.r2.ensure(vb);
  w.p2.ensure(vb);
  cplx<T> *rB = w.r2.as<cplx<T>>(), *pB = w.p2.as<cplx<T>>();
  auto compact = [&]() {
    const int nnew = nact + (nact & 1);
    w.cidx.ensure(sizeof(int) * (size_t)n);
    w.cd.ensure(sizeof(double) * 5 * 2 * (size_t)n);
    w.ci.ensure(sizeof(int) * 6 * 2 * (size_t)n);
    const int set = nset == 1 ? 2 : 1;
    double *dd = w.cd.as<double>() + (size_t)(set - 1) * 5 * n;
    int *di = w.ci.as<int>() + (size_t)(set - 1) * 6 * n;
    CgRows nx{dd, dd + n, dd + 2 * (size_t)n, dd + 3 * (size_t)n, learned ? dd + 4 * (size_t)n : nullptr,
              di, di + n, di + 2 * (size_t)n, learned ? di + 3 * (size_t)n : nullptr, learned ? di + 4 * (size_t)n : nullptr,
              di + 5 * (size_t)n};
    int *src = w.cidx.as<int>();
    if (nset > 0)  // counts (and TPA-fallback rows) of the solves about to be dropped
      launch("compact", 0, k_scatter_home, dim3((ncur + 127) / 128), dim3(128), 0, st, cur, ncur, ii + n,
             learned ? c->krow.as<int>() : nullptr);
    launch("compact", 0, k_compact_index, dim3(1), dim3(1024), 0, st, (const int *)cur.active, ncur, src);
    launch("compact", 0, k_compact_scalars, dim3((nnew + 127) / 128), dim3(128), 0, st, cur, nx, (const int *)src, nnew, nact);
    launch("compact", bits_of<T>(), k_compact_vectors<T>, dim3(grid_for((size_t)nnew * g.ld)), dim3(256), 0, st, g,
           (const cplx<T> *)r, (const cplx<T> *)p, rB, pB, (const int *)src, nnew, nact);
    WDF_CUDA_TRY(cudaGetLastError());
    std::swap(r, rB);
    std::swap(p, pB);
    cur = nx;
    ncur = nnew;
    nset = set;
    s.rz = cur.rz;
    s.rz_new = cur.rz_new;
    s.thr = cur.thr;
    s.shift = cur.shift;
    s.active = cur.active;
    s.iters = cur.iters;
    s.vidx = cur.krow;
    s.home = cur.home;
    if (learned) {
      s.krow = cur.krow;
      s.vorig = cur.vorig;
      s.rr_ref = cur.rr_ref;
      s.it_ref = cur.it_ref;
    }
  };
  PDir<T> dir;
  dir.K = K;
  for (int it = 0; it < maxiter && nact > 0; ++it) {
    if (compaction && nact <= ncur - std::max(8, ncur / 8)) compact();
    dir.p = p;
    dir.r = r;
    dir.vidx = s.vidx;
    dir.active = s.active;
    dir.beta = s.rz_new;
    // p = K r + beta p (from the second iteration on), A p and the partial sums of <p, A p>
    int ndot = apply_operator_cg<T>(c, p, Ap, ncur, s.shift, it > 0 ? &dir : nullptr, s.part1);
    if (ndot == 0) {
      launch_dot_partial<T>(g, p, Ap, ncur, s.part1, nch, st);
      ndot = nch;
    }
    launch_cg_scalars(s, ncur, ndot, 0, maxiter, st);
    launch_cg_update<T>(g, x, r, nullptr, p, Ap, K, s, ncur, nch, st);
    WDF_CUDA_TRY(cudaMemsetAsync(s.nactive, 0, sizeof(int), st));
    launch_cg_scalars(s, ncur, nch, 1, maxiter, st);
    WDF_CUDA_TRY(cudaMemcpyAsync(&nact, s.nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
    WDF_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (nset > 0) {
    launch("compact", 0, k_scatter_home, dim3((ncur + 127) / 128), dim3(128), 0, st, cur, ncur, ii + n,
           learned ? c->krow.as<int>() : nullptr);
    WDF_CUDA_TRY(cudaGetLastError());
  }
  iters.resize(n);
  WDF_CUDA_TRY(cudaMemcpyAsync(iters.data(), ii + n, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  WDF_CUDA_TRY(cudaStreamSynchronize(st));
}

void apply_sternheimer_operator(wdf_ctx *c, const cplx<double> *X, cplx<double> *Y, const int *vidx_host, int n) {
  if (n <= 0) return;
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  c->vidx_dev.ensure(sizeof(int) * n);
  c->shift.ensure(sizeof(double) * n);
  WDF_CUDA_TRY(cudaMemcpyAsync(c->vidx_dev.p, vidx_host, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  launch("gather_shift", 0, k_gather_shift, dim3((n + 127) / 128), dim3(128), 0, st, c->vidx_dev.as<int>(), c->eps_dev.as<double>(),
         c->shift.as<double>(), n);
  WDF_CUDA_TRY(cudaGetLastError());
  if (c->opt.precision == WDF_MIXED_DF) {
    const size_t vb = sizeof(cplx<double>) * (size_t)n * g.ld;
    c->dfa.ensure(vb);
    c->dfb.ensure(vb);
    to_df(c, c->dfa.as<cplx<df64>>(), X, n);
    apply_operator<df64>(c, c->dfa.as<cplx<df64>>(), c->dfb.as<cplx<df64>>(), n, c->shift.as<double>(), true);
    from_df(c, Y, c->dfb.as<cplx<df64>>(), n);
  } else {
    apply_operator<double>(c, X, Y, n, c->shift.as<double>(), true);
  }
  int terr = 0;
  WDF_CUDA_TRY(cudaMemcpyAsync(&terr, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  WDF_CUDA_TRY(cudaStreamSynchronize(st));
  if (terr) throw ApiFailure(WDF_ETIMEOUT, "a kernel gave up waiting for its MMAs or bulk copies");
}

// FP64 outer loop: r = b - A x in FP64, inner solve A d = r (FP64 or FP32), x += d.
void sternheimer_solve(wdf_ctx *c, const cplx<double> *b, cplx<double> *x, const int *vidx_host, int n, SolveStats &ss) {
  if (n <= 0) return;
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  const bool mixed = c->opt.precision != WDF_FP64;  // FP32 inner solves (WDF_MIXED, WDF_MIXED_DF)
  const size_t vb = sizeof(cplx<double>) * (size_t)n * g.ld;
  c->vidx_dev.ensure(sizeof(int) * n);
  c->shift.ensure(sizeof(double) * n);
  c->thr.ensure(sizeof(double) * n);
  WDF_CUDA_TRY(cudaMemcpyAsync(c->vidx_dev.p, vidx_host, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  launch("gather_shift", 0, k_gather_shift, dim3((n + 127) / 128), dim3(128), 0, st, c->vidx_dev.as<int>(), c->eps_dev.as<double>(), c->shift.as<double>(), n);
  WDF_CUDA_TRY(cudaGetLastError());
  c->rr.ensure(vb);
  c->rAx.ensure(vb);
  cplx<double> *r = c->rr.as<cplx<double>>(), *Ax = c->rAx.as<cplx<double>>();
  double *nrm = c->dv_small.as<double>();
  c->dv_small.ensure(sizeof(double) * 2 * (size_t)n);
  nrm = c->dv_small.as<double>();
  dots<double>(c, b, b, n, nrm);
  const std::vector<double> bb = to_host(c, nrm, n);
  const bool learned = c->opt.precond == WDF_PRECOND_LEARNED;
  if (learned) {
    if (!c->has_model) throw ApiFailure(WDF_EINVAL, "WDF_PRECOND_LEARNED without a model (wdf_set_model)");
    c->krow.ensure(sizeof(int) * n);
    c->rr_ref.ensure(sizeof(double) * n);
    c->it_ref.ensure(sizeof(int) * n);
    c->nfb.ensure(sizeof(int));
    WDF_CUDA_TRY(cudaMemcpyAsync(c->krow.p, c->vidx_dev.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    WDF_CUDA_TRY(cudaMemsetAsync(c->nfb.p, 0, sizeof(int), st));
  }
  // r = b - A x; A x in FP64, or in double-float (FP64 vectors converted in and out)
  auto residual = [&]() {
    if (c->opt.precision == WDF_MIXED_DF) {
      c->dfa.ensure(vb);
      c->dfb.ensure(vb);
      to_df(c, c->dfa.as<cplx<df64>>(), x, n);
      apply_operator<df64>(c, c->dfa.as<cplx<df64>>(), c->dfb.as<cplx<df64>>(), n, c->shift.as<double>(), true);
      from_df(c, Ax, c->dfb.as<cplx<df64>>(), n);
    } else {
      apply_operator<double>(c, x, Ax, n, c->shift.as<double>(), true);
    }
    WDF_CUDA_TRY(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, st));
    launch_axpby<double>(g, r, Ax, n, -1.0, 1.0, st);
  };
  // Residual updates (FP32 inner forms). The residual of x + d is r - A d exactly; once the
  // correction d is small, A d in FP32 is accurate enough: its error is at most eps_A ||d||, with
  // eps_A measured on this batch (16 x the largest ||A x - A_32 x|| / ||x|| over its solves, at the
  // first iterate, A x in the residual precision). A refinement takes r - A_32 d when every
  // solve's accumulated bound stays below tol ||b|| / 10, else the full residual; the stopping
  // test and the reported residual add the bound to ||r||. Only with opt.residual_update set;
  // otherwise every refinement recomputes b - A x in the residual precision.
  const bool may_update = mixed && c->opt.residual_update != 0;
  double epsA = -1.0;
  std::vector<double> bnd(n, 0.0);
  auto calibrate = [&]() {
    auto &w = c->cg32;
    w.x.ensure(sizeof(cplx<float>) * (size_t)n * g.ld);
    c->rwork.ensure(sizeof(cplx<float>) * (size_t)n * g.ld);
    cplx<float> *x32 = c->rwork.as<cplx<float>>(), *y32 = w.x.as<cplx<float>>();
    launch_convert<double, float>(g, (float *)x32, (const double *)x, 2 * (size_t)n * g.ld, st);
    apply_operator<float>(c, x32, y32, n, c->shift.as<double>(), true);
    const int nch = dot_chunks(g);
    c->cg64.part1.ensure(sizeof(double) * (size_t)n * nch);
    launch_diff_partial(g, Ax, y32, n, c->cg64.part1.as<double>(), nch, st);
    launch("sum_chunks", 0, k_sum_chunks, dim3((n + 127) / 128), dim3(128), 0, st, c->cg64.part1.as<double>(), n, nch, nrm + n);
    WDF_CUDA_TRY(cudaGetLastError());
    const std::vector<double> dev2 = to_host(c, nrm + n, n);
    dots<double>(c, x, x, n, nrm + n);
    const std::vector<double> xx = to_host(c, nrm + n, n);
    epsA = 0.0;
    for (int s = 0; s < n; ++s)
      if (xx[s] > 0.0) epsA = std::max(epsA, std::sqrt(dev2[s] / xx[s]));
    epsA *= 16.0;
    if (!std::isfinite(epsA)) epsA = -1.0;
  };
  if (learned && c->opt.warm_start) {  // x0 = o1 K b from the model, then its residual
    launch_first_iterate(g, x, b, c->mlw64.as<double>(), c->vidx_dev.as<int>(), n, st);
    residual();
  } else {
    WDF_CUDA_TRY(cudaMemsetAsync(x, 0, vb, st));
    WDF_CUDA_TRY(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, st));
  }
  const double tol = c->opt.cg_tol;
  const int maxref = mixed ? 12 : 6;
  std::vector<int> iters_total(n, 0), it;
  std::vector<double> rr(n, 0.0);
  std::vector<double> thr(n);
  bool conv = false;
  ss.refinements = 0;
  const bool trace = std::getenv("WDF_TRACE") != nullptr;
  for (int ref = 0; ref <= maxref; ++ref) {
    dots<double>(c, r, r, n, nrm);
    rr = to_host(c, nrm, n);
    int nact = 0, nunconv = 0;
    double worst = 0.0;
    for (int s = 0; s < n; ++s) {
      const double rn = std::sqrt(rr[s]) + bnd[s];  // a bound on ||b - A x||
      const bool unconv = bb[s] > 0.0 && rn * rn > tol * tol * bb[s];
      const bool act = unconv && iters_total[s] < c->opt.cg_maxiter;
      if (!std::isfinite(rr[s])) throw ApiFailure(WDF_ENAN, "non-finite residual in a Sternheimer solve");
      if (unconv) ++nunconv;
      if (bb[s] > 0.0) worst = std::max(worst, rn / std::sqrt(bb[s]));
      if (act) {
        ++nact;
        double eta = 0.5 * tol * std::sqrt(bb[s] / rr[s]);
        if (mixed) eta = std::max(eta, c->opt.inner_tol);
        eta = std::max(eta, 1e-15);
        thr[s] = eta * eta * rr[s];
      } else {
        thr[s] = 1e300;  // start inactive
      }
    }
    if (trace) {
      int itmax = 0;
      for (int s = 0; s < n; ++s) itmax = std::max(itmax, iters_total[s]);
      fprintf(stderr, "[wdf] refinement %d: %d of %d solves above tol, worst rel residual %.3e, max iterations %d\n", ref,
              nunconv, n, worst, itmax);
    }
    if (nunconv == 0) {
      conv = true;
      break;
    }
    if (nact == 0) break;  // iteration budget spent
    if (ref == maxref) break;
    ss.refinements = ref + 1;
    bool updated = false;
    WDF_CUDA_TRY(cudaMemcpyAsync(c->thr.p, thr.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    int budget = 0;
    for (int s = 0; s < n; ++s) budget = std::max(budget, c->opt.cg_maxiter - iters_total[s]);
    if (mixed) {
      auto &w = c->cg32;
      w.x.ensure(sizeof(cplx<float>) * (size_t)n * g.ld);
      c->rwork.ensure(sizeof(cplx<float>) * (size_t)n * g.ld);
      cplx<float> *r32 = c->rwork.as<cplx<float>>(), *d32 = w.x.as<cplx<float>>();
      launch_convert<double, float>(g, (float *)r32, (const double *)r, 2 * (size_t)n * g.ld, st);
      cg_solve<float>(c, r32, d32, n, budget, it);
      // x += d ; reuse Ax as FP64 staging of d
      launch_convert<float, double>(g, (double *)Ax, (const float *)d32, 2 * (size_t)n * g.ld, st);
      launch_axpby<double>(g, x, Ax, n, 1.0, 1.0, st);
      if (epsA >= 0.0 && may_update) {  // r - A_32 d when every bound stays small
        dots<double>(c, Ax, Ax, n, nrm + n);
        const std::vector<double> dd = to_host(c, nrm + n, n);
        std::vector<double> cand(n);
        updated = true;
        for (int s = 0; s < n; ++s) {
          cand[s] = bnd[s] + epsA * std::sqrt(dd[s]);
          if (bb[s] > 0.0 && cand[s] > 0.1 * tol * std::sqrt(bb[s])) updated = false;
        }
        if (updated) {
          bnd = cand;
          apply_operator<float>(c, d32, r32, n, c->shift.as<double>(), true);
          launch_convert<float, double>(g, (double *)Ax, (const float *)r32, 2 * (size_t)n * g.ld, st);
          launch_axpby<double>(g, r, Ax, n, -1.0, 1.0, st);
        }
      }
    } else {
      auto &w = c->cg64;
      w.x.ensure(vb);
      cplx<double> *d = w.x.as<cplx<double>>();
      cg_solve<double>(c, r, d, n, budget, it);
      launch_axpby<double>(g, x, d, n, 1.0, 1.0, st);
    }
    for (int s = 0; s < n; ++s) iters_total[s] += it[s];
    if (trace) fprintf(stderr, "[wdf] refinement %d: %s residual (eps_A %.3e)\n", ref, updated ? "updated" : "full", epsA);
    if (!updated) {
      residual();
      std::fill(bnd.begin(), bnd.end(), 0.0);
      if (may_update && epsA < 0.0) calibrate();
    }
  }
  {
    int terr = 0;
    WDF_CUDA_TRY(cudaMemcpyAsync(&terr, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    WDF_CUDA_TRY(cudaStreamSynchronize(st));
    if (terr) throw ApiFailure(WDF_ETIMEOUT, "a kernel gave up waiting for its MMAs or bulk copies");
  }
  ss.converged = conv;
  ss.fallbacks = 0;
  if (learned) {
    WDF_CUDA_TRY(cudaMemcpyAsync(&ss.fallbacks, c->nfb.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    WDF_CUDA_TRY(cudaStreamSynchronize(st));
  }
  ss.iters = 0;
  ss.iters_max = 0;
  ss.max_res = 0.0;
  for (int s = 0; s < n; ++s) {
    ss.iters += iters_total[s];
    ss.iters_max = std::max(ss.iters_max, iters_total[s]);
    if (bb[s] > 0) ss.max_res = std::max(ss.max_res, (std::sqrt(rr[s]) + bnd[s]) / std::sqrt(bb[s]));
  }
}

// ---------------------------------------------------------------------------------------------
// chi0bar by DFPT (paper Sec. 2.1). phi: npert internal FP64 vectors (G = 0 ignored).

// Stages S2, S3, S7, S8 in R (FP64 or double-float); xp: np2 rows of v^1/2 phi (FP64). Results
// (np2 rows, FP64) go to ou = v^1/2 drho and dr = drho.
template <typename R>
static void chi0_stages(wdf_ctx *c, const cplx<double> *xp64, int npert, const std::vector<char> &zero, cplx<double> *ou,
                        cplx<double> *dr, SolveStats &ss) {
  constexpr bool DF = std::is_same<R, df64>::value;
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  const FftCtx<R> &f = Prec<R>::f(c);
  wdf_ctx::Cg &w = Prec<R>::cg(c);
  const int npp = (npert + 1) / 2, np2 = 2 * npp, nocc = c->nocc;
  const size_t ngrid = c->ngrid;
  const size_t cbpair = (size_t)g.n3 * g.ldcb;
  const size_t rowb = sizeof(cplx<R>) * g.ld;
  const cplx<R> *xp;
  if constexpr (DF) {
    c->xpdf.ensure(rowb * np2);
    to_df(c, c->xpdf.as<cplx<df64>>(), xp64, np2);
    xp = c->xpdf.as<cplx<R>>();
  } else {
    xp = xp64;
  }
  // dV pairs in real space: dV_2pp + i dV_2pp+1 = ifft(x_2pp + i x_2pp+1)
  DBuf &dvb = Stage<R>::dv(c);
  dvb.ensure(sizeof(cplx<R>) * (size_t)npp * ngrid);
  cplx<R> *dv = dvb.as<cplx<R>>();
  {
    w.cb.ensure(sizeof(cplx<R>) * (size_t)npp * cbpair);
    launch_zpass_g2r<R>(f, xp, np2, w.cb.as<cplx<R>>(), st);
    PlaneArgs<R> pa;
    pa.cb = w.cb.as<cplx<R>>();
    pa.grid = dv;
    launch_plane<R>(f, OP_G2R, npp, pa, st);
  }
  cplx<R> *drR, *ouR;
  if constexpr (DF) {
    c->drdf.ensure(rowb * np2);
    c->oudf.ensure(rowb * np2);
    drR = c->drdf.as<cplx<R>>();
    ouR = c->oudf.as<cplx<R>>();
  } else {
    drR = dr;
    ouR = ou;
  }
  // perturbation pairs per chunk so that at most max_batch solves are resident
  int cpp = npp;
  if (c->opt.max_batch > 0) cpp = std::max(1, std::min(npp, c->opt.max_batch / (2 * nocc)));
  ss = SolveStats();
  SolveStats sc;
  const cplx<R> *psi = Prec<R>::U(c) + (size_t)c->nproj * g.ld;
  for (int pp0 = 0; pp0 < npp; pp0 += cpp) {
    const int pp1 = std::min(npp, pp0 + cpp);
    const int nq = (pp1 - pp0) * nocc, ns = 2 * nq;
    // right-hand sides b_vp = -Q fft_n(dV_p psi_v)
    c->rb.ensure(sizeof(cplx<double>) * (size_t)ns * g.ld);
    c->rx.ensure(sizeof(cplx<double>) * (size_t)ns * g.ld);
    cplx<double> *b = c->rb.as<cplx<double>>(), *x = c->rx.as<cplx<double>>();
    cplx<R> *bR;
    if constexpr (DF) {
      c->dfa.ensure(rowb * ns);
      bR = c->dfa.as<cplx<R>>();
    } else {
      bR = b;
    }
    w.cb.ensure(sizeof(cplx<R>) * (size_t)nq * cbpair);
    cplx<R> *cb = w.cb.as<cplx<R>>();
    {
      PlaneArgs<R> pa;
      pa.cb = cb;
      pa.field = Stage<R>::psir(c);
      pa.grid = dv + (size_t)pp0 * ngrid;
      pa.nocc = nocc;
      launch_plane<R>(f, OP_PROD_R2G, nq, pa, st);
      EpiArgs<R> ea;
      ea.Y = bR;
      ea.scale = R(1.0 / (double)ngrid);
      launch_zpass_r2g<R>(f, EPI_STORE, cb, ns, ea, st);
      w.S.ensure(sizeof(double) * (size_t)nocc * ns);
      bool done = false;
      if constexpr (DF) {
        if (c->oz_on) {  // b = -(b - psi (psi^T b)) on the tensor cores
          oz_lowrank(c, c->nproj, nocc, c->oz_pt, bR, bR, ns, nullptr, -1.f, w.S.as<double>());
          done = true;
        }
      }
      if (!done) {
        gram<R>(c, psi, nocc, bR, ns, w.S.as<double>(), ns);
        launch_lincomb<R>(g, bR, ns, psi, nocc, w.S.as<double>(), ns, nullptr, -1.0, st);
      }
      if constexpr (DF) from_df(c, b, bR, ns);
    }
    // a perturbation that is zero (and the phantom partner of an odd last one) has a right-hand
    // side of FFT rounding noise from its Gamma partner: set it to exactly zero so that its
    // solves are skipped and its response is zero
    const size_t row = sizeof(cplx<double>) * g.ld;
    for (int p = 2 * pp0; p < 2 * pp1; ++p)
      if (p >= npert || zero[p])
        WDF_CUDA_TRY(cudaMemset2DAsync(b + ((size_t)2 * (p / 2 - pp0) * nocc + (p & 1)) * g.ld, 2 * row, 0, row, nocc, st));
    std::vector<int> vidx(ns);
    for (int s = 0; s < ns; ++s) vidx[s] = (s / 2) % nocc;
    sternheimer_solve(c, b, x, vidx.data(), ns, sc);
    if (c->collect) launch_mlp_accum(g, b, x, ns, nocc, c->kp64.as<double>(), c->mlsums.as<double>(), st);
    ss.fallbacks += sc.fallbacks;
    ss.iters += sc.iters;
    ss.iters_max = std::max(ss.iters_max, sc.iters_max);
    ss.refinements = std::max(ss.refinements, sc.refinements);
    ss.max_res = std::max(ss.max_res, sc.max_res);
    ss.converged = ss.converged && sc.converged;
    // drho_p = (4/Omega) fft_n(sum_v psi_v ifft(dpsi_vp)); out = v^1/2 drho
    const cplx<R> *xR;
    if constexpr (DF) {
      c->dfb.ensure(rowb * ns);
      to_df(c, c->dfb.as<cplx<df64>>(), x, ns);
      xR = c->dfb.as<cplx<R>>();
    } else {
      xR = x;
    }
    w.cb.ensure(sizeof(cplx<R>) * (size_t)nq * cbpair);
    cb = w.cb.as<cplx<R>>();
    DBuf &cb2 = Stage<R>::cb2(c), &accb = Stage<R>::acc(c);
    cb2.ensure(sizeof(cplx<R>) * (size_t)(pp1 - pp0) * cbpair);
    accb.ensure(sizeof(cplx<R>) * (size_t)(pp1 - pp0) * ngrid);
    launch_zpass_g2r<R>(f, xR, ns, cb, st);
    if (plane_accum_by_g2r<R>(f)) {
      // per perturbation pair: every orbital's pair to real space (compile-time plane kernel), then
      // the sum over orbitals on the grid; then the summed grids back to their column buffers
      // (the product kernel with psi = 1)
      DBuf &fields = Stage<R>::fields(c), &ones = Stage<R>::ones(c);
      fields.ensure(sizeof(cplx<R>) * (size_t)nocc * ngrid);
      if (ones.cap < sizeof(R) * ngrid) {
        ones.ensure(sizeof(R) * ngrid);
        launch_fill<R>(ones.as<R>(), ngrid, 1.0, st);
      }
      for (int pp = pp0; pp < pp1; ++pp) {
        PlaneArgs<R> pg;
        pg.cb = cb + (size_t)(pp - pp0) * nocc * cbpair;
        pg.grid = fields.as<cplx<R>>();
        launch_plane<R>(f, OP_G2R, nocc, pg, st);
        launch_orbital_sum<R>(fields.as<cplx<R>>(), Stage<R>::psir(c), nocc, ngrid, accb.as<cplx<R>>() + (size_t)(pp - pp0) * ngrid, st);
      }
      PlaneArgs<R> pb;
      pb.cb = cb2.as<cplx<R>>();
      pb.field = ones.as<R>();
      pb.grid = accb.as<cplx<R>>();
      pb.nocc = 1;
      launch_plane<R>(f, OP_PROD_R2G, pp1 - pp0, pb, st);
    } else {
      PlaneArgs<R> pa;
      pa.cb = cb;
      pa.cb2 = cb2.as<cplx<R>>();
      pa.field = Stage<R>::psir(c);
      pa.grid = accb.as<cplx<R>>();
      pa.nocc = nocc;
      launch_plane<R>(f, OP_ACCUM, pp1 - pp0, pa, st);
    }
    EpiArgs<R> ea;
    ea.Y = drR + (size_t)(2 * pp0) * g.ld;
    ea.Y2 = ouR + (size_t)(2 * pp0) * g.ld;
    ea.vhalf = c->t_vhalf.as<double>();
    ea.scale = R(4.0 / (c->omega * (double)ngrid));
    launch_zpass_r2g<R>(f, EPI_DRHO, cb2.as<cplx<R>>(), 2 * (pp1 - pp0), ea, st);
  }
  if constexpr (DF) {
    from_df(c, dr, drR, np2);
    from_df(c, ou, ouR, np2);
  }
}

void chi0_apply_internal(wdf_ctx *c, const cplx<double> *phi, int npert, cplx<double> *out, cplx<double> *drho,
                         SolveStats &ss) {
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  const int npp = (npert + 1) / 2, np2 = 2 * npp;
  // x = v^1/2 phi (extra zero row when npert is odd)
  c->xpert.ensure(sizeof(cplx<double>) * (size_t)np2 * g.ld);
  cplx<double> *xp = c->xpert.as<cplx<double>>();
  WDF_CUDA_TRY(cudaMemsetAsync(xp, 0, sizeof(cplx<double>) * (size_t)np2 * g.ld, st));
  launch("scale_elems", 0, k_scale_elems, dim3(grid_for((size_t)npert * g.ld)), dim3(256), 0, st, g, xp, phi,
         c->t_vhalf.as<double>(), npert);
  WDF_CUDA_TRY(cudaGetLastError());
  // results go to scratch with an even number of rows (the last pair may hold a phantom row)
  c->chi_out.ensure(sizeof(cplx<double>) * (size_t)np2 * g.ld);
  c->chi_drho.ensure(sizeof(cplx<double>) * (size_t)np2 * g.ld);
  cplx<double> *dr = c->chi_drho.as<cplx<double>>(), *ou = c->chi_out.as<cplx<double>>();
  // perturbations that are exactly zero
  std::vector<char> zero(npert, 0);
  {
    c->pnorm.ensure(sizeof(double) * (size_t)npert);
    dots<double>(c, xp, xp, npert, c->pnorm.as<double>());
    const std::vector<double> n2 = to_host(c, c->pnorm.as<double>(), npert);
    for (int p = 0; p < npert; ++p) zero[p] = n2[p] == 0.0;
  }
  if (c->opt.precision == WDF_MIXED_DF) chi0_stages<df64>(c, xp, npert, zero, ou, dr, ss);
  else chi0_stages<double>(c, xp, npert, zero, ou, dr, ss);
  const size_t nb = sizeof(cplx<double>) * (size_t)npert * g.ld;
  WDF_CUDA_TRY(cudaMemcpyAsync(out, ou, nb, cudaMemcpyDeviceToDevice, st));
  if (drho) WDF_CUDA_TRY(cudaMemcpyAsync(drho, dr, nb, cudaMemcpyDeviceToDevice, st));
}

// ---------------------------------------------------------------------------------------------
// low-rank W_p from PDEP eigenpairs (Eq. 5 without the Xi term)

void wp_apply_internal(wdf_ctx *c, const cplx<double> *phib, const double *coef, int neig, const cplx<double> *x, int nvec,
                       cplx<double> *y) {
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  c->wp_vx.ensure(sizeof(cplx<double>) * (size_t)nvec * g.ld);
  c->wp_S.ensure(sizeof(double) * (size_t)neig * nvec);
  cplx<double> *vx = c->wp_vx.as<cplx<double>>();
  const double *vh = c->t_vhalf.as<double>();
  // v^1/2 x; S_a = <phibar_a, v^1/2 x>; y = sum_a phibar_a coef_a S_a; W_p x = v^1/2 y
  launch("scale_elems", 0, k_scale_elems, dim3(grid_for((size_t)nvec * g.ld)), dim3(256), 0, st, g, vx, x, vh, nvec);
  WDF_CUDA_TRY(cudaGetLastError());
  gram<double>(c, phib, neig, vx, nvec, c->wp_S.as<double>(), nvec);
  WDF_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(cplx<double>) * (size_t)nvec * g.ld, st));
  launch_lincomb<double>(g, y, nvec, phib, neig, c->wp_S.as<double>(), nvec, coef, 0.0, st);
  launch("scale_elems", 0, k_scale_elems, dim3(grid_for((size_t)nvec * g.ld)), dim3(256), 0, st, g, y, (const cplx<double> *)y, vh,
         nvec);
  WDF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// block Davidson

static void copy_rows(wdf_ctx *c, cplx<double> *dst, const cplx<double> *src, int n) {
  if (n <= 0 || dst == src) return;
  WDF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(cplx<double>) * (size_t)n * c->geo.ld, cudaMemcpyDeviceToDevice, c->st));
}

// Make rows [nb, nb + nnew) of V orthonormal to rows [0, nb) and to each other: unit scaling,
// two passes of block classical Gram-Schmidt against the old rows, then vector by vector (two
// passes) within the block; vectors left with norm < drop are removed. Returns the number kept
// (compacted to rows nb ...).
static int orthonormalise(wdf_ctx *c, cplx<double> *V, int nb, int nnew, double drop) {
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  if (nnew <= 0) return 0;
  cplx<double> *Nw = V + (size_t)nb * g.ld;
  double *sm = c->dv_small.as<double>();
  double *neg = c->dv_neg.as<double>();
  // unit scaling
  dots<double>(c, Nw, Nw, nnew, sm);
  std::vector<double> n2 = to_host(c, sm, nnew);
  std::vector<double> inv(nnew);
  for (int i = 0; i < nnew; ++i) inv[i] = n2[i] > 0 ? 1.0 / std::sqrt(n2[i]) : 0.0;
  WDF_CUDA_TRY(cudaMemcpyAsync(sm, inv.data(), sizeof(double) * nnew, cudaMemcpyHostToDevice, st));
  launch_scale_rows<double>(g, Nw, sm, nnew, st);
  double *C = c->dv_Y.as<double>();  // scratch nb x nnew
  for (int pass = 0; pass < 2 && nb > 0; ++pass) {
    gram<double>(c, V, nb, Nw, nnew, C, nnew);
    launch_lincomb<double>(g, Nw, nnew, V, nb, C, nnew, neg, 1.0, st);
  }
  // within the block: CholeskyQR2 (Gram matrix, Cholesky, N <- N L^-T, twice) when the block is
  // well conditioned; near-dependent blocks take the vector-by-vector path below, which drops
  if (nnew > 1 && nnew <= kCholMax) {
    const size_t nn = (size_t)nnew * nnew;
    c->chol.ensure(sizeof(double) * 2 * nn + sizeof(int));
    c->rwork.ensure(sizeof(cplx<double>) * (size_t)nnew * g.ld);
    double *Gm = c->chol.as<double>(), *Cf = Gm + nn;
    int *ok = reinterpret_cast<int *>(Cf + nn);
    cplx<double> *tmp = c->rwork.as<cplx<double>>();
    int good = 1;
    for (int pass = 0; pass < 2 && good; ++pass) {
      gram<double>(c, Nw, nnew, Nw, nnew, Gm, nnew);
      // CholeskyQR squares the condition number: accept pivots above 1e-12 of the largest
      launch_chol_inv(Gm, nnew, Cf, pass == 0 ? 1e-12 : 0.25, ok, st);
      WDF_CUDA_TRY(cudaMemcpyAsync(&good, ok, sizeof(int), cudaMemcpyDeviceToHost, st));
      WDF_CUDA_TRY(cudaStreamSynchronize(st));
      if (!good) break;
      launch_lincomb<double>(g, tmp, nnew, Nw, nnew, Cf, nnew, nullptr, 0.0, st);
      // the lincomb writes elements [0, nint) of each row; the padding of Nw stays as it was
      const size_t row = sizeof(cplx<double>) * (size_t)g.ld;
      WDF_CUDA_TRY(cudaMemcpy2DAsync(Nw, row, tmp, row, sizeof(cplx<double>) * (size_t)g.nint, nnew, cudaMemcpyDeviceToDevice, st));
    }
    if (good) return nnew;
    // fall back: the block may have lost orthogonality in the first pass; the sequential path
    // below re-orthonormalises from the current vectors
  }
  int kept = 0;
  for (int i = 0; i < nnew; ++i) {
    cplx<double> *vi = Nw + (size_t)i * g.ld;
    cplx<double> *base = Nw;  // kept rows are Nw[0 .. kept)
    for (int pass = 0; pass < 2 && kept > 0; ++pass) {
      gram<double>(c, base, kept, vi, 1, C, 1);
      launch_lincomb<double>(g, vi, 1, base, kept, C, 1, neg, 1.0, st);
    }
    dots<double>(c, vi, vi, 1, sm);
    const double nn = std::sqrt(to_host(c, sm, 1)[0]);
    if (!(nn >= drop)) continue;
    const double s = 1.0 / nn;
    WDF_CUDA_TRY(cudaMemcpyAsync(sm, &s, sizeof(double), cudaMemcpyHostToDevice, st));
    launch_scale_rows<double>(g, vi, sm, 1, st);
    copy_rows(c, Nw + (size_t)kept * g.ld, vi, 1);
    ++kept;
  }
  return kept;
}

DavResult davidson(wdf_ctx *c, DavOp &op, const cplx<double> *V0, int n0, int nwant, int nkeep, int nbmax, int maxiter,
                   double tol, bool zero_g0) {
  (void)zero_g0;
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  DavResult res;
  // after a restart the basis holds nkeep Ritz vectors plus at most nkeep new ones
  nbmax = std::max(nbmax, 2 * nkeep);
  const size_t vb = sizeof(cplx<double>) * (size_t)g.ld;
  c->dv_V.ensure(vb * (size_t)std::max(nbmax, n0));
  c->dv_W.ensure(vb * (size_t)std::max(nbmax, n0));
  c->dv_X.ensure(vb * (size_t)nkeep);
  c->dv_AX.ensure(vb * (size_t)nkeep);
  c->dv_R.ensure(vb * (size_t)nkeep);
  c->dv_H.ensure(sizeof(double) * (size_t)nbmax * nbmax);
  c->dv_Y.ensure(sizeof(double) * (size_t)std::max(nbmax, n0) * std::max(nbmax, n0));
  c->dv_theta.ensure(sizeof(double) * nbmax);
  c->dv_jac.ensure(sizeof(double) * jacobi_work_doubles(nbmax));
  set_jacobi_limits(nbmax);
  c->dv_jint.ensure(sizeof(int) * 4);
  WDF_CUDA_TRY(cudaMemsetAsync(c->dv_jint.p, 0, sizeof(int) * 4, st));
  c->dv_small.ensure(sizeof(double) * (size_t)std::max(nbmax, n0) * 2);
  c->dv_neg.ensure(sizeof(double) * (size_t)std::max(nbmax, n0));
  {
    std::vector<double> neg(std::max(nbmax, n0), -1.0);
    WDF_CUDA_TRY(cudaMemcpyAsync(c->dv_neg.p, neg.data(), sizeof(double) * neg.size(), cudaMemcpyHostToDevice, st));
  }
  cplx<double> *V = c->dv_V.as<cplx<double>>(), *W = c->dv_W.as<cplx<double>>();
  cplx<double> *X = c->dv_X.as<cplx<double>>(), *AX = c->dv_AX.as<cplx<double>>(), *R = c->dv_R.as<cplx<double>>();
  double *H = c->dv_H.as<double>(), *Y = c->dv_Y.as<double>(), *theta = c->dv_theta.as<double>();
  const double drop = 1e-12;
  copy_rows(c, V, V0, n0);
  int nb = orthonormalise(c, V, 0, n0, drop);
  if (nb < nkeep) throw ApiFailure(WDF_EINVAL, "start block has fewer independent vectors than requested eigenpairs");
  if (nb > nbmax) nb = nbmax;
  op.apply(V, W, nb);
  res.napply = nb;
  std::vector<double> th, rn;
  for (int it = 1; it <= maxiter; ++it) {
    res.iters = it;
    gram<double>(c, V, nb, W, nb, H, nb);
    jacobi_eigh(H, Y, theta, nb, c->dv_jac.as<double>(), c->dv_jint.as<int>(), st, c->wait_polls);
    const int k = std::min(nkeep, nb);
    launch_lincomb<double>(g, X, k, V, nb, Y, nb, nullptr, 0.0, st);
    launch_lincomb<double>(g, AX, k, W, nb, Y, nb, nullptr, 0.0, st);
    launch_ritz_residual(g, R, AX, X, theta, k, st);
    dots<double>(c, R, R, k, c->dv_small.as<double>());
    rn = to_host(c, c->dv_small.as<double>(), k);
    th = to_host(c, theta, k);
    {  // the eigensolve's grid barrier gives up (and flags it) instead of waiting forever
      int jerr = 0;
      WDF_CUDA_TRY(cudaMemcpyAsync(&jerr, c->dv_jint.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
      WDF_CUDA_TRY(cudaStreamSynchronize(st));
      if (jerr) throw ApiFailure(WDF_ETIMEOUT, "the subspace eigensolver gave up waiting at a grid barrier");
    }
    bool all = true;
    std::vector<int> unconv;
    for (int a = 0; a < k; ++a) {
      rn[a] = std::sqrt(std::max(0.0, rn[a]));
      const bool ok = rn[a] <= tol;
      if (!ok) unconv.push_back(a);
      if (a < nwant && !ok) all = false;
    }
    res.lam = th;
    res.resnorm = rn;
    if (all) {
      res.converged = true;
      break;
    }
    if (it == maxiter) break;
    const int nu = (int)unconv.size();
    if (nb + nu > nbmax) {  // restart from the Ritz vectors
      copy_rows(c, V, X, k);
      copy_rows(c, W, AX, k);
      nb = k;
    }
    cplx<double> *Nw = V + (size_t)nb * g.ld;
    for (int i = 0; i < nu; ++i) copy_rows(c, Nw + (size_t)i * g.ld, R + (size_t)unconv[i] * g.ld, 1);
    if (op.precondition()) {
      // TPA with the kinetic energy of each Ritz vector
      double *tk = c->dv_small.as<double>();
      c->rwork.ensure(sizeof(double) * (size_t)nu * g.ld);
      for (int i = 0; i < nu; ++i) launch_kinetic(g, X + (size_t)unconv[i] * g.ld, 1, tk + i, st);
      launch_tpa_table<double>(g, c->rwork.as<double>(), tk, nu, st);
      launch_mul_table<double>(g, Nw, c->rwork.as<double>(), nu, st);
    }
    const int kept = orthonormalise(c, V, nb, nu, drop);
    if (kept == 0) break;
    op.apply(Nw, W + (size_t)nb * g.ld, kept);
    res.napply += kept;
    nb += kept;
  }
  return res;
}

// ---------------------------------------------------------------------------------------------
// ground state of H (paper Eq. (1)) by the same Davidson, TPA-preconditioned

struct HamOp : DavOp {
  wdf_ctx *c;
  explicit HamOp(wdf_ctx *cc) : c(cc) {}
  void apply(const cplx<double> *X, cplx<double> *Y, int n) override { apply_operator<double>(c, X, Y, n, nullptr, false); }
  bool precondition() const override { return true; }
};

void ground_state(wdf_ctx *c) {
  const Geo &g = c->geo;
  const Layout &L = c->lay;
  const int nev = std::min(c->nocc + std::max(0, c->opt.gs_extra), 2 * L.nint - L.len0);
  // start block: the plane waves of lowest kinetic energy as cos / sin pairs (no random numbers)
  std::vector<int> order;
  for (int e = 0; e < L.nint; ++e) {
    if (L.e_col[e] == 0 && L.e_z[e] < 0) continue;  // column (0,0): one of each +-z pair
    order.push_back(e);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return L.g2[a] < L.g2[b]; });
  const int n0 = nev;
  std::vector<cplx<double>> h0((size_t)n0 * g.ld, mkc<double>(0, 0));
  int made = 0;
  for (size_t t = 0; t < order.size() && made < n0; ++t) {
    const int e = order[t];
    const bool self = (L.e_col[e] == 0 && L.e_z[e] == 0);
    for (int kind = 0; kind < (self ? 1 : 2) && made < n0; ++kind) {
      cplx<double> *v = h0.data() + (size_t)made * g.ld;
      v[e] = kind == 0 ? mkc<double>(1, 0) : mkc<double>(0, 1);
      if (L.e_col[e] == 0 && L.e_z[e] > 0) {  // mirror inside column (0,0)
        const int e2 = L.col_off[0] + (-L.e_z[e] - L.col_zlo[0]);
        v[e2] = kind == 0 ? mkc<double>(1, 0) : mkc<double>(0, -1);
      }
      ++made;
    }
  }
  c->rx.ensure(sizeof(cplx<double>) * h0.size());
  WDF_CUDA_TRY(cudaMemcpyAsync(c->rx.p, h0.data(), sizeof(cplx<double>) * h0.size(), cudaMemcpyHostToDevice, c->st));
  WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
  HamOp op(c);
  DavResult r = davidson(c, op, c->rx.as<cplx<double>>(), n0, c->nocc, nev, 3 * nev, c->opt.gs_maxiter, c->opt.gs_tol, false);
  c->eps.assign(r.lam.begin(), r.lam.begin() + c->nocc);
  c->gap = (nev > c->nocc) ? r.lam[c->nocc] - r.lam[c->nocc - 1] : 0.0;
  copy_rows(c, c->U64.as<cplx<double>>() + (size_t)c->nproj * g.ld, c->dv_X.as<cplx<double>>(), c->nocc);
  WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (!r.converged) throw ApiFailure(WDF_ENOCONV, "ground state Davidson did not converge");
}

// tables that depend on the occupied orbitals
// time the V_loc plane variants (register, Stockham, generic, persistent) on a zero column buffer
// of 128 pairs (enough units for the persistent kernel's pipeline to fill) and keep the fastest in
// f.vloc_variant
template <typename T> static void autotune_vloc(wdf_ctx *c, FftCtx<T> &f, const T *vloc) {
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  const int nblk = 128;
  const size_t bytes = sizeof(cplx<T>) * (size_t)nblk * g.n3 * g.ldcb;
  DBuf cbuf;
  cbuf.ensure(bytes);
  WDF_CUDA_TRY(cudaMemsetAsync(cbuf.p, 0, bytes, st));
  PlaneArgs<T> pa;
  pa.cb = cbuf.as<cplx<T>>();
  pa.field = vloc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 1e30f;
  int bestv = 0;
  if (const char *pin = std::getenv("WDF_PLANE_VARIANT")) {  // fixed choice, e.g. to compare contexts bit for bit
    const int v = std::atoi(pin);
    if (v >= 1 && v <= kPlaneVariants && plane_variant_available<T>(f, v)) {
      f.vloc_variant = v;
      cbuf.release();
      return;
    }
  }
  try {
    WDF_CUDA_TRY(cudaEventCreate(&e0));
    WDF_CUDA_TRY(cudaEventCreate(&e1));
    for (int v = 1; v <= kPlaneVariants; ++v) {
      if (!plane_variant_available<T>(f, v)) continue;
      f.vloc_variant = v;
      launch_plane<T>(f, OP_VLOC, nblk, pa, st);  // warm-up
      WDF_CUDA_TRY(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) launch_plane<T>(f, OP_VLOC, nblk, pa, st);
      WDF_CUDA_TRY(cudaEventRecord(e1, st));
      WDF_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      WDF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (std::getenv("WDF_TRACE")) fprintf(stderr, "[wdf]   plane variant %d (%d-bit): %.3f ms per %d pairs\n", v, bits_of<T>(), ms / 3, nblk);
      if (ms < best) {
        best = ms;
        bestv = v;
      }
    }
  } catch (...) {
    if (e0) (void)cudaEventDestroy(e0);
    if (e1) (void)cudaEventDestroy(e1);
    cbuf.release();
    throw;
  }
  (void)cudaEventDestroy(e0);
  (void)cudaEventDestroy(e1);
  cbuf.release();
  f.vloc_variant = bestv;
  if (std::getenv("WDF_TRACE"))
    fprintf(stderr, "[wdf] V_loc plane kernel (%d-bit): variant %d (1 register, 2 Stockham, 3 generic, 4 two-thread register, 5 persistent, 6 double-float, 7 two-thread persistent), %.3f ms per %d pairs\n",
            bits_of<T>(), bestv, best / 3, nblk);
}

void finish_setup(wdf_ctx *c) {
  const Geo &g = c->geo;
  cudaStream_t st = c->st;
  const int nocc = c->nocc, M = c->nproj + nocc;
  double emin = c->eps[0], emax = c->eps[0];
  for (double e : c->eps) {
    emin = std::min(emin, e);
    emax = std::max(emax, e);
  }
  c->alpha = c->opt.alpha > 0 ? c->opt.alpha : (emax - emin + 1.0);
  std::vector<double> lrd(M);
  for (int j = 0; j < c->nproj; ++j) lrd[j] = c->dij[j];
  for (int v = 0; v < nocc; ++v) lrd[c->nproj + v] = c->alpha;
  c->lrd.ensure(sizeof(double) * M);
  WDF_CUDA_TRY(cudaMemcpyAsync(c->lrd.p, lrd.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
  c->eps_dev.ensure(sizeof(double) * nocc);
  WDF_CUDA_TRY(cudaMemcpyAsync(c->eps_dev.p, c->eps.data(), sizeof(double) * nocc, cudaMemcpyHostToDevice, st));
  const cplx<double> *psi = c->U64.as<cplx<double>>() + (size_t)c->nproj * g.ld;
  // psi_v(r) = ifft_u(c_v), two orbitals per complex transform
  const int npair = (nocc + 1) / 2;
  c->psir64.ensure(sizeof(double) * (size_t)nocc * c->ngrid);
  c->psir32.ensure(sizeof(float) * (size_t)nocc * c->ngrid);
  c->accgrid.ensure(sizeof(cplx<double>) * (size_t)npair * c->ngrid);
  c->cg64.cb.ensure(sizeof(cplx<double>) * (size_t)npair * g.n3 * g.ldcb);
  launch_zpass_g2r<double>(c->f64, psi, nocc, c->cg64.cb.as<cplx<double>>(), st);
  PlaneArgs<double> pa;
  pa.cb = c->cg64.cb.as<cplx<double>>();
  pa.grid = c->accgrid.as<cplx<double>>();
  launch_plane<double>(c->f64, OP_G2R, npair, pa, st);
  launch("split_pairs", 64, k_split_pairs<double>, dim3(grid_for((size_t)npair * c->ngrid)), dim3(256), 0, st, c->accgrid.as<cplx<double>>(), npair, c->ngrid,
                                                                           c->psir64.as<double>(), nocc);
  WDF_CUDA_TRY(cudaGetLastError());
  launch_convert<double, float>(g, c->psir32.as<float>(), c->psir64.as<double>(), (size_t)nocc * c->ngrid, st);
  // TPA tables
  c->tkin.ensure(sizeof(double) * nocc);
  launch_kinetic(g, psi, nocc, c->tkin.as<double>(), st);
  c->kp64.ensure(sizeof(double) * (size_t)nocc * g.ld);
  c->kp32.ensure(sizeof(float) * (size_t)nocc * g.ld);
  launch_tpa_table<double>(g, c->kp64.as<double>(), c->tkin.as<double>(), nocc, st);
  launch_tpa_table<float>(g, c->kp32.as<float>(), c->tkin.as<double>(), nocc, st);
  // FP32 copy of the projectors and orbitals
  c->U32.ensure(sizeof(cplx<float>) * (size_t)M * g.ld);
  launch_convert<double, float>(g, (float *)c->U32.p, (const double *)c->U64.p, 2 * (size_t)M * g.ld, st);
  // tensor-core copies of U for the FP32 projections (the Gram runs in chunks of 256 rows of U, the
  // linear combination in K chunks of 32, so any height up to kTcMaxRows)
  // one device flag for every kernel with a bounded wait (tensor-core MMAs, bulk copies)
  c->tcerr.ensure(sizeof(int));
  WDF_CUDA_TRY(cudaMemsetAsync(c->tcerr.p, 0, sizeof(int), st));
  c->f32.err = c->tcerr.as<int>();
  c->tc_on = tc_enabled() && M >= 1 && M <= kTcMaxRows;
  if (c->tc_on) {
    const int kp = tc_rows(M);
    c->tcU.ensure(sizeof(float) * 2 * (size_t)M * 2 * g.ld);
    c->tcUt.ensure(sizeof(float) * 2 * (size_t)2 * g.ld * kp);
    launch_tc_prep_u(g, c->U32.as<float2>(), M, c->tc_uwh(), c->tc_uwl(), c->tc_uth(), c->tc_utl(), st);
  }
  if (c->opt.precision == WDF_MIXED_DF) {  // double-float copies for residuals and density
    c->Udf.ensure(sizeof(cplx<df64>) * (size_t)M * g.ld);
    to_df(c, c->Udf.as<cplx<df64>>(), c->U64.as<cplx<double>>(), M);
    c->vlocdf.ensure(sizeof(df64) * c->ngrid);
    launch_convert<double, df64>(g, c->vlocdf.as<df64>(), c->vloc64.as<double>(), c->ngrid, st);
    c->psirdf.ensure(sizeof(df64) * (size_t)nocc * c->ngrid);
    launch_convert<double, df64>(g, c->psirdf.as<df64>(), c->psir64.as<double>(), (size_t)nocc * c->ngrid, st);
    // digits of the weighted rows of U (the Gram's A operand), of U^T over all rows and of psi^T
    // over the orbital rows (the linear combinations' B operands), from the FP64 copy
    c->oz_on = oz_enabled() && c->tc_on;
    if (c->oz_on) {
      const int kf = 2 * g.nint;
      c->oz_u = oz_mat(c->ozU, c->ozUe, M, kf);
      launch_oz_rows_f64(g, c->U64.as<cplx<double>>(), M, true, c->oz_u, st);
      c->oz_ut = oz_mat(c->ozUt, c->ozUte, kf, M);
      launch_oz_cols(c->U64.as<double>(), (size_t)2 * g.ld, M, kf, nullptr, c->oz_ut, st);
      c->oz_pt = oz_mat(c->ozPt, c->ozPte, kf, nocc);
      launch_oz_cols(c->U64.as<double>() + (size_t)c->nproj * 2 * g.ld, (size_t)2 * g.ld, nocc, kf, nullptr, c->oz_pt, st);
    }
  }
  // the V_loc plane kernels of the inner CG and of the residuals: time the variants that exist
  // for this grid and keep the fastest
  autotune_vloc<float>(c, c->f32, c->vloc32.as<float>());
  if (c->opt.precision == WDF_MIXED_DF) autotune_vloc<df64>(c, c->fdf, c->vlocdf.as<df64>());
  else autotune_vloc<double>(c, c->f64, c->vloc64.as<double>());
  WDF_CUDA_TRY(cudaStreamSynchronize(st));
}

template void apply_operator<double>(wdf_ctx *, const cplx<double> *, cplx<double> *, int, const double *, bool);
template void apply_operator<float>(wdf_ctx *, const cplx<float> *, cplx<float> *, int, const double *, bool);
template void apply_operator<df64>(wdf_ctx *, const cplx<df64> *, cplx<df64> *, int, const double *, bool);

}  // namespace wdf

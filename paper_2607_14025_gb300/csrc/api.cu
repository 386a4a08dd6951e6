// C ABI entry points of libwdf.so (declared in include/wdf.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "engine.cuh"

using namespace wdf;

namespace wdf {
static thread_local std::string g_last_error;
void set_error(int, const std::string &msg) { g_last_error = msg; }
const char *last_global_error() { return g_last_error.c_str(); }

thread_local Profiler *t_prof = nullptr;
std::atomic<long long> g_launches{0};

void prof_record(cudaStream_t st) {
  Profiler *p = t_prof;
  if (p->used == p->ev.size()) {
    cudaEvent_t e;
    WDF_CUDA_TRY(cudaEventCreate(&e));
    p->ev.push_back(e);
  }
  WDF_CUDA_TRY(cudaEventRecord(p->ev[p->used++], st));
}
}  // namespace wdf

namespace {

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double ms() const { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
};

template <class F> int guarded(wdf_ctx *c, F &&body) {
  if (c && c->failed) {
    c->err = "context unusable after an earlier CUDA failure";
    return WDF_ESTATE;
  }
  struct ProfScope {  // kernel timing applies to launches made inside this call only
    explicit ProfScope(wdf_ctx *c) { t_prof = (c && c->prof_on) ? &c->prof : nullptr; }
    ~ProfScope() { t_prof = nullptr; }
  } scope(c);
  try {
    if (c) {
      cudaError_t e = cudaSetDevice(c->device);
      if (e != cudaSuccess) throw CudaFailure(e, "cudaSetDevice", __FILE__, __LINE__);
    }
    return body();
  } catch (const ApiFailure &f) {
    if (c) c->err = f.msg;
    set_error(f.code, f.msg);
    return f.code;
  } catch (const CudaFailure &f) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(f.err), cudaGetErrorString(f.err), f.what,
             f.file, f.line);
    if (c) {
      c->err = buf;
      c->failed = true;
    }
    set_error(WDF_ECUDA, buf);
    return WDF_ECUDA;
  } catch (const std::bad_alloc &) {
    if (c) c->err = "host allocation failed";
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  } catch (...) {
    if (c) c->err = "unexpected C++ exception";
    set_error(WDF_EINVAL, "unexpected C++ exception");
    return WDF_EINVAL;
  }
}

void check_mem(int mem) {
  if (mem != WDF_MEM_HOST && mem != WDF_MEM_DEVICE) throw ApiFailure(WDF_EINVAL, "mem must be WDF_MEM_HOST or WDF_MEM_DEVICE");
}

// Bring external (caller) half-sphere data into device memory: returns a device pointer to
// n * npw_h complex values (the caller's pointer itself for device memory).
const double *stage_in(wdf_ctx *c, DBuf &buf, const double *src, size_t ndouble, int mem) {
  if (mem == WDF_MEM_DEVICE) return src;
  buf.ensure(ndouble * sizeof(double));
  WDF_CUDA_TRY(cudaMemcpyAsync(buf.p, src, ndouble * sizeof(double), cudaMemcpyHostToDevice, c->st));
  return buf.as<double>();
}

// copy internal FP64 vectors out to the caller in external layout
void write_out(wdf_ctx *c, DBuf &stage, const cplx<double> *in, int n, double *dst, int mem) {
  const size_t nd = 2 * (size_t)n * c->npw_h;
  double *target = dst;
  if (mem == WDF_MEM_HOST) {
    stage.ensure(nd * sizeof(double));
    target = stage.as<double>();
  }
  launch_int_to_ext(in, n, c->geo.ld, c->npw_h, c->t_emap.as<int>(), c->t_econj.as<int>(), target, c->st);
  if (mem == WDF_MEM_HOST) WDF_CUDA_TRY(cudaMemcpyAsync(dst, target, nd * sizeof(double), cudaMemcpyDeviceToHost, c->st));
}

// external -> internal FP64 (into buf), optional per-element scale
cplx<double> *read_in(wdf_ctx *c, DBuf &stage, DBuf &buf, const double *src, int n, int mem, int extra_rows = 0) {
  const double *d = stage_in(c, stage, src, 2 * (size_t)n * c->npw_h, mem);
  const size_t bytes = sizeof(cplx<double>) * (size_t)(n + extra_rows) * c->geo.ld;
  buf.ensure(bytes);
  WDF_CUDA_TRY(cudaMemsetAsync(buf.p, 0, bytes, c->st));
  launch_ext_to_int(d, n, c->npw_h, c->t_emap.as<int>(), c->t_emap2.as<int>(), c->t_econj.as<int>(), nullptr,
                    buf.as<cplx<double>>(), c->geo.ld, c->st);
  return buf.as<cplx<double>>();
}

template <class T> void upload(wdf_ctx *c, DBuf &b, const std::vector<T> &h) {
  b.ensure(std::max<size_t>(1, h.size()) * sizeof(T));
  if (!h.empty()) WDF_CUDA_TRY(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
}

void fill_stats(wdf_stats *st, const SolveStats &ss, long long nsolve, long long napply, double ms) {
  if (!st) return;
  memset(st, 0, sizeof *st);
  st->nsolve = nsolve;
  st->cg_iters = ss.iters;
  st->cg_iters_max = ss.iters_max;
  st->refinements = ss.refinements;
  st->max_residual = ss.max_res;
  st->napply = napply;
  st->converged = ss.converged ? 1 : 0;
  st->ms = ms;
}

void setup_body(wdf_ctx *c, const wdf_system *sys) {
  check_mem(sys->mem);
  if (!sys->miller || !sys->vloc_r) throw ApiFailure(WDF_EINVAL, "miller and vloc_r are required");
  if (sys->nproj < 0 || (sys->nproj > 0 && (!sys->beta || !sys->dij))) throw ApiFailure(WDF_EINVAL, "nproj > 0 needs beta and dij");
  if (sys->nocc < 1) throw ApiFailure(WDF_EINVAL, "nocc must be at least 1");
  if ((sys->psi == nullptr) != (sys->eps == nullptr)) throw ApiFailure(WDF_EINVAL, "psi and eps must be given together");
  for (int a = 0; a < 3; ++a) c->n[a] = sys->n[a];
  memcpy(c->cell, sys->cell, sizeof c->cell);
  // reciprocal vectors b_i (rows) with a_i . b_j = 2 pi delta_ij: B = 2 pi (A^-1)^T
  const double *A = c->cell;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 0)) throw ApiFailure(WDF_EINVAL, "singular cell");
  c->omega = std::fabs(det);
  const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det, (A[1] * A[5] - A[2] * A[4]) / det,
                         (A[5] * A[6] - A[3] * A[8]) / det, (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det, (A[0] * A[4] - A[1] * A[3]) / det};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c->bvec[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
  c->npw_h = sys->npw_h;
  c->nproj = sys->nproj;
  c->nocc = sys->nocc;
  c->lay = build_layout(sys->miller, sys->npw_h, sys->n, c->bvec);
  const Layout &L = c->lay;
  if (2 * L.nint - L.len0 <= c->nocc) throw ApiFailure(WDF_EINVAL, "more occupied orbitals than plane waves");
  c->ngrid = (size_t)sys->n[0] * sys->n[1] * sys->n[2];
  if (sys->nproj > 0) c->dij.assign(sys->dij, sys->dij + sys->nproj);

  // device tables
  upload(c, c->t_col_off, L.col_off);
  upload(c, c->t_col_zlo, L.col_zlo);
  upload(c, c->t_e_col, L.e_col);
  upload(c, c->t_e_z, L.e_z);
  upload(c, c->t_tile, L.tile_idx);
  upload(c, c->t_xact, L.xact);
  upload(c, c->t_xactn, L.xactn);
  upload(c, c->t_jidx, L.jidx);
  upload(c, c->t_pos3, L.pos3);
  upload(c, c->t_g2, L.g2);
  upload(c, c->t_vhalf, L.vhalf);
  upload(c, c->t_emap, L.emap);
  upload(c, c->t_emap2, L.emap2);
  upload(c, c->t_econj, L.econj);
  // twiddles exp(2 pi i t / n) from long double sines and cosines
  std::vector<double> tw64;
  std::vector<float> tw32;
  for (int a = 0; a < 3; ++a) {
    for (int t = 0; t < kMaxN; ++t) {
      long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)sys->n[a];
      double cr = t < sys->n[a] ? (double)cosl(ang) : 0.0, ci = t < sys->n[a] ? (double)sinl(ang) : 0.0;
      tw64.push_back(cr);
      tw64.push_back(ci);
      tw32.push_back((float)cr);
      tw32.push_back((float)ci);
    }
  }
  upload(c, c->t_tw64, tw64);
  upload(c, c->t_tw32, tw32);
  {
    std::vector<df64> twdf(tw64.size());
    for (size_t i = 0; i < tw64.size(); ++i) twdf[i] = df64(tw64[i]);
    upload(c, c->t_twdf, twdf);
  }

  Geo &g = c->geo;
  g.n1 = sys->n[0];
  g.n2 = sys->n[1];
  g.n3 = sys->n[2];
  g.pitch = g.n1 + 1;
  g.K = L.K;
  g.ndisk = L.ndisk;
  g.ldcb = L.ldcb;
  g.nint = L.nint;
  g.ld = L.ld;
  g.len0 = L.len0;
  g.nxact = (int)L.xact.size();
  g.col_off = c->t_col_off.as<int>();
  g.col_zlo = c->t_col_zlo.as<int>();
  g.e_col = c->t_e_col.as<int>();
  g.e_z = c->t_e_z.as<int>();
  g.tile_idx = c->t_tile.as<int>();
  g.xact = c->t_xact.as<int>();
  g.xactn = c->t_xactn.as<int>();
  g.xmax = L.xmax;
  g.pos3 = c->t_pos3.as<short>();
  g.g2 = c->t_g2.as<double>();
  c->f64.g = g;
  c->f32.g = g;
  c->f64.P1 = c->f32.P1 = L.P1;
  c->f64.P2 = c->f32.P2 = L.P2;
  c->f64.P3 = c->f32.P3 = L.P3;
  const cplx<double> *t64 = c->t_tw64.as<cplx<double>>();
  const cplx<float> *t32 = c->t_tw32.as<cplx<float>>();
  c->fdf.g = g;
  c->fdf.P1 = L.P1;
  c->fdf.P2 = L.P2;
  c->fdf.P3 = L.P3;
  {
    const cplx<df64> *tdf = c->t_twdf.as<cplx<df64>>();
    c->fdf.tw1 = tdf;
    c->fdf.tw2 = tdf + kMaxN;
    c->fdf.tw3 = tdf + 2 * kMaxN;
  }
  c->f64.jidx = c->f32.jidx = c->fdf.jidx = (std::getenv("WDF_GENERIC_PLANE") ? nullptr : c->t_jidx.as<int>());
  c->f64.tw1 = t64;
  c->f64.tw2 = t64 + kMaxN;
  c->f64.tw3 = t64 + 2 * kMaxN;
  c->f32.tw1 = t32;
  c->f32.tw2 = t32 + kMaxN;
  c->f32.tw3 = t32 + 2 * kMaxN;
  if (plane_smem<double>(g) > 227 * 1024 || zpass_smem<double>(g) > 227 * 1024)
    throw ApiFailure(WDF_EINVAL, "FFT plane does not fit in shared memory in FP64 (n1 * n2 too large)");
  set_fft_smem_limits<double>(g);
  set_fft_smem_limits<float>(g);
  set_fft_smem_limits<df64>(g);

  // local potential
  c->vloc64.ensure(sizeof(double) * c->ngrid);
  c->vloc32.ensure(sizeof(float) * c->ngrid);
  WDF_CUDA_TRY(cudaMemcpyAsync(c->vloc64.p, sys->vloc_r, sizeof(double) * c->ngrid,
                               sys->mem == WDF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
  launch_convert<double, float>(g, c->vloc32.as<float>(), c->vloc64.as<double>(), c->ngrid, c->st);
  // projectors and orbitals in internal layout: U64 rows [beta; psi]
  const int M = c->nproj + c->nocc;
  c->U64.ensure(sizeof(cplx<double>) * (size_t)M * g.ld);
  WDF_CUDA_TRY(cudaMemsetAsync(c->U64.p, 0, sizeof(cplx<double>) * (size_t)M * g.ld, c->st));
  if (c->nproj > 0) {
    const double *d = stage_in(c, c->ext_in, sys->beta, 2 * (size_t)c->nproj * c->npw_h, sys->mem);
    launch_ext_to_int(d, c->nproj, c->npw_h, c->t_emap.as<int>(), c->t_emap2.as<int>(), c->t_econj.as<int>(), nullptr,
                      c->U64.as<cplx<double>>(), g.ld, c->st);
  }
  c->lrd.ensure(sizeof(double) * M);
  {
    std::vector<double> lrd(M, 0.0);
    for (int j = 0; j < c->nproj; ++j) lrd[j] = c->dij[j];
    WDF_CUDA_TRY(cudaMemcpyAsync(c->lrd.p, lrd.data(), sizeof(double) * M, cudaMemcpyHostToDevice, c->st));
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  c->flag.ensure(sizeof(int));
  WDF_CUDA_TRY(cudaMemsetAsync(c->flag.p, 0, sizeof(int), c->st));
  launch_check_finite<double>(c->vloc64.as<double>(), c->ngrid, c->flag.as<int>(), c->st);
  launch_check_finite<double>((const double *)c->U64.p, 2 * (size_t)c->nproj * g.ld, c->flag.as<int>(), c->st);
  int bad = 0;
  WDF_CUDA_TRY(cudaMemcpyAsync(&bad, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (bad) throw ApiFailure(WDF_ENAN, "non-finite value in vloc_r or beta");
  int status = WDF_OK;
  if (sys->psi) {
    const double *d = stage_in(c, c->ext_in, sys->psi, 2 * (size_t)c->nocc * c->npw_h, sys->mem);
    launch_ext_to_int(d, c->nocc, c->npw_h, c->t_emap.as<int>(), c->t_emap2.as<int>(), c->t_econj.as<int>(), nullptr,
                      c->U64.as<cplx<double>>() + (size_t)c->nproj * g.ld, g.ld, c->st);
    c->eps.assign(sys->eps, sys->eps + c->nocc);
    for (double e : c->eps)
      if (!std::isfinite(e)) throw ApiFailure(WDF_ENAN, "non-finite eigenvalue");
  } else {
    try {
      ground_state(c);
    } catch (const ApiFailure &f) {
      if (f.code != WDF_ENOCONV) throw;
      c->err = f.msg;
      status = WDF_ENOCONV;
    }
  }
  finish_setup(c);
  if (status != WDF_OK) throw ApiFailure(status, c->err);
}

struct Chi0Op : DavOp {
  wdf_ctx *c;
  SolveStats agg;
  long long nsolve = 0;
  explicit Chi0Op(wdf_ctx *cc) : c(cc) {}
  void apply(const cplx<double> *X, cplx<double> *Y, int n) override {
    SolveStats ss;
    chi0_apply_internal(c, X, n, Y, nullptr, ss);
    agg.iters += ss.iters;
    agg.iters_max = std::max(agg.iters_max, ss.iters_max);
    agg.refinements = std::max(agg.refinements, ss.refinements);
    agg.max_res = std::max(agg.max_res, ss.max_res);
    agg.converged = agg.converged && ss.converged;
    nsolve += (long long)n * c->nocc;
  }
};

}  // namespace

extern "C" {

void wdf_default_options(wdf_options *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = WDF_MIXED;
  o->precond = WDF_PRECOND_TPA;
  o->cg_tol = 1e-8;
  o->cg_maxiter = 1000;
  o->inner_tol = 1e-5;
  o->alpha = 0.0;
  o->max_batch = 0;
  o->gs_tol = 1e-10;
  o->gs_maxiter = 300;
  o->gs_extra = 8;
  o->stream = nullptr;
  o->device = 0;
}

int wdf_setup_hamiltonian(wdf_ctx **out, const wdf_system *sys, const wdf_options *opt) {
  if (!out || !sys) {
    set_error(WDF_EINVAL, "out and sys must not be NULL");
    return WDF_EINVAL;
  }
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    set_error(WDF_ESTATE, "no CUDA device available");
    return WDF_ESTATE;
  }
  wdf_ctx *c = new (std::nothrow) wdf_ctx();
  if (!c) {
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  }
  if (opt) c->opt = *opt;
  else wdf_default_options(&c->opt);
  if (c->opt.device < 0 || c->opt.device >= ndev) {
    delete c;
    set_error(WDF_EINVAL, "device ordinal out of range");
    return WDF_EINVAL;
  }
  if ((c->opt.precision != WDF_FP64 && c->opt.precision != WDF_MIXED && c->opt.precision != WDF_MIXED_DF) ||
      (c->opt.precond != WDF_PRECOND_NONE && c->opt.precond != WDF_PRECOND_TPA) || !(c->opt.cg_tol > 0) ||
      c->opt.cg_maxiter < 1 || !(c->opt.inner_tol > 0 && c->opt.inner_tol < 1) || !(c->opt.gs_tol > 0) || c->opt.gs_maxiter < 1 ||
      c->opt.max_batch < 0 || c->opt.gs_extra < 0) {
    delete c;
    set_error(WDF_EINVAL, "invalid option value");
    return WDF_EINVAL;
  }
  c->device = c->opt.device;
  c->st = (cudaStream_t)c->opt.stream;
  int rc = guarded(c, [&] {
    setup_body(c, sys);
    return WDF_OK;
  });
  if (rc != WDF_OK && rc != WDF_ENOCONV) {
    set_error(rc, c->err);
    wdf_destroy(c);
    return rc;
  }
  *out = c;
  return rc;
}

void wdf_destroy(wdf_ctx *c) {
  if (!c) return;
  (void)cudaSetDevice(c->device);
  if (c->st) (void)cudaStreamSynchronize(c->st);
  else (void)cudaDeviceSynchronize();
  DBuf *bufs[] = {&c->t_col_off, &c->t_col_zlo, &c->t_e_col, &c->t_e_z,   &c->t_tile,  &c->t_xact,   &c->t_pos3,   &c->t_g2,
                  &c->t_vhalf,   &c->t_emap,    &c->t_emap2, &c->t_econj, &c->t_tw64,  &c->t_tw32,   &c->vloc64,   &c->vloc32,
                  &c->U64,       &c->U32,       &c->lrd,     &c->psir64,  &c->psir32,  &c->kp64,     &c->kp32,     &c->tkin,
                  &c->eps_dev,   &c->rb,        &c->rx,      &c->rr,      &c->rAx,     &c->rwork,    &c->shift,    &c->vidx_dev,
                  &c->thr,       &c->gramw,     &c->xpert,   &c->dvgrid,  &c->accgrid, &c->cb2,      &c->outi,     &c->drhoi,
                  &c->ext_in,    &c->ext_out,   &c->ext_out2, &c->dv_V,   &c->dv_W,    &c->dv_X,     &c->dv_AX,    &c->dv_R,
                  &c->dv_H,      &c->dv_Y,      &c->dv_theta, &c->dv_jac, &c->dv_jint, &c->dv_small, &c->dv_neg,   &c->zeros,
                  &c->flag,      &c->guess,     &c->chi_out, &c->chi_drho, &c->t_xactn, &c->t_jidx,
                  &c->t_twdf,    &c->vlocdf,    &c->Udf,     &c->psirdf,   &c->dfa,     &c->dfb,
                  &c->xpdf,      &c->dvgriddf,  &c->accgriddf, &c->cb2df,  &c->drdf,    &c->oudf};
  for (DBuf *b : bufs) b->release();
  for (cudaEvent_t e : c->prof.ev) (void)cudaEventDestroy(e);
  for (wdf_ctx::Cg *w : {&c->cg64, &c->cg32, &c->cgdf}) {
    DBuf *cb[] = {&w->r, &w->z, &w->p, &w->Ap, &w->x, &w->cb, &w->S, &w->part1, &w->part2, &w->dbl, &w->ints};
    for (DBuf *b : cb) b->release();
  }
  delete c;
}

int wdf_get_orbitals(wdf_ctx *c, double *eps, double *psi, int mem) {
  if (!c || !eps) return WDF_EINVAL;
  return guarded(c, [&] {
    check_mem(mem);
    memcpy(eps, c->eps.data(), sizeof(double) * c->nocc);
    if (psi) {
      write_out(c, c->ext_out, c->U64.as<cplx<double>>() + (size_t)c->nproj * c->geo.ld, c->nocc, psi, mem);
      WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    return WDF_OK;
  });
}

int wdf_apply_hamiltonian(wdf_ctx *c, int nvec, const double *in, double *out, int mem) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    check_mem(mem);
    if (nvec < 0 || (nvec > 0 && (!in || !out))) throw ApiFailure(WDF_EINVAL, "bad nvec or NULL buffer");
    if (nvec == 0) return WDF_OK;
    cplx<double> *X = read_in(c, c->ext_in, c->xpert, in, nvec, mem);
    c->outi.ensure(sizeof(cplx<double>) * (size_t)nvec * c->geo.ld);
    apply_operator<double>(c, X, c->outi.as<cplx<double>>(), nvec, nullptr, false);
    write_out(c, c->ext_out, c->outi.as<cplx<double>>(), nvec, out, mem);
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    return WDF_OK;
  });
}

int wdf_sternheimer(wdf_ctx *c, int nsolve, const int32_t *vidx, const double *rhs, double *x, int mem, wdf_stats *st) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    Timer tm;
    check_mem(mem);
    if (nsolve < 0 || (nsolve > 0 && (!vidx || !rhs || !x))) throw ApiFailure(WDF_EINVAL, "bad nsolve or NULL buffer");
    for (int s = 0; s < nsolve; ++s)
      if (vidx[s] < 0 || vidx[s] >= c->nocc) throw ApiFailure(WDF_EINVAL, "vidx out of range");
    SolveStats ss;
    if (nsolve > 0) {
      cplx<double> *B = read_in(c, c->ext_in, c->rb, rhs, nsolve, mem);
      c->rx.ensure(sizeof(cplx<double>) * (size_t)nsolve * c->geo.ld);
      std::vector<int> v(vidx, vidx + nsolve);
      sternheimer_solve(c, B, c->rx.as<cplx<double>>(), v.data(), nsolve, ss);
      write_out(c, c->ext_out, c->rx.as<cplx<double>>(), nsolve, x, mem);
      WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    fill_stats(st, ss, nsolve, 0, tm.ms());
    return ss.converged ? WDF_OK : WDF_ENOCONV;
  });
}

int wdf_apply_chi0(wdf_ctx *c, int npert, const double *phi, double *out, double *drho, int mem, wdf_stats *st) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    Timer tm;
    check_mem(mem);
    if (npert < 0 || (npert > 0 && (!phi || !out))) throw ApiFailure(WDF_EINVAL, "bad npert or NULL buffer");
    SolveStats ss;
    if (npert > 0) {
      cplx<double> *P = read_in(c, c->ext_in, c->guess, phi, npert, mem, 1);
      const int np2 = 2 * ((npert + 1) / 2);
      c->outi.ensure(sizeof(cplx<double>) * (size_t)np2 * c->geo.ld);
      c->drhoi.ensure(sizeof(cplx<double>) * (size_t)np2 * c->geo.ld);
      chi0_apply_internal(c, P, npert, c->outi.as<cplx<double>>(), c->drhoi.as<cplx<double>>(), ss);
      write_out(c, c->ext_out, c->outi.as<cplx<double>>(), npert, out, mem);
      if (drho) write_out(c, c->ext_out2, c->drhoi.as<cplx<double>>(), npert, drho, mem);
      WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    fill_stats(st, ss, (long long)npert * c->nocc, npert, tm.ms());
    return ss.converged ? WDF_OK : WDF_ENOCONV;
  });
}

int wdf_pdep_davidson(wdf_ctx *c, int neig, int nbasis_max, int maxiter, double tol, int nguess, const double *guess,
                      double *lambda, double *phibar, int mem, wdf_stats *st) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    Timer tm;
    check_mem(mem);
    if (neig < 1 || nguess < neig || !guess || !lambda || !phibar || maxiter < 1 || !(tol > 0) || nbasis_max < 0)
      throw ApiFailure(WDF_EINVAL, "bad Davidson arguments");
    if (neig > 2 * c->geo.nint - c->geo.len0 - 1) throw ApiFailure(WDF_EINVAL, "neig exceeds the basis dimension");
    const int nbmax = nbasis_max > 0 ? nbasis_max : 4 * neig;
    cplx<double> *G0 = read_in(c, c->ext_in, c->guess, guess, nguess, mem);
    // perturbations carry no G = 0 component (element -zlo of column (0,0))
    const int e0 = c->lay.col_off[0] - c->lay.col_zlo[0];
    WDF_CUDA_TRY(cudaMemset2DAsync(G0 + e0, sizeof(cplx<double>) * c->geo.ld, 0, sizeof(cplx<double>), nguess, c->st));
    Chi0Op op(c);
    DavResult r = davidson(c, op, G0, nguess, neig, neig, nbmax, maxiter, tol, true);
    for (int a = 0; a < neig; ++a) lambda[a] = r.lam[a];
    write_out(c, c->ext_out, c->dv_X.as<cplx<double>>(), neig, phibar, mem);
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    op.agg.converged = op.agg.converged && r.converged;
    fill_stats(st, op.agg, op.nsolve, r.napply, tm.ms());
    if (st) st->davidson_iters = r.iters;
    return r.converged ? WDF_OK : WDF_ENOCONV;
  });
}

int wdf_profile_kernel(wdf_ctx *c, const char *kernel) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    if (c->st) WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    c->prof.used = 0;
    c->prof.count = 0;
    c->prof_on = kernel != nullptr;
    if (!kernel) return WDF_OK;
    std::string k(kernel);
    int bits = 0;
    const size_t colon = k.find(':');
    if (colon != std::string::npos) {
      bits = std::atoi(k.c_str() + colon + 1);
      k = k.substr(0, colon);
      if (bits != 32 && bits != 64 && bits != 48) throw ApiFailure(WDF_EINVAL, "kernel precision suffix must be :32, :48 or :64");
    }
    c->prof.target = k;
    c->prof.bits = bits;
    return WDF_OK;
  });
}

int wdf_profile_read(wdf_ctx *c, int64_t *launches, double *ms) {
  if (!c || !launches || !ms) return WDF_EINVAL;
  return guarded(c, [&] {
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->prof.used; i += 2) {
      float t = 0.f;
      WDF_CUDA_TRY(cudaEventElapsedTime(&t, c->prof.ev[i], c->prof.ev[i + 1]));
      tot += t;
    }
    *launches = c->prof.count;
    *ms = tot;
    return WDF_OK;
  });
}

int64_t wdf_launch_count(void) { return (int64_t)g_launches.load(); }

const char *wdf_strerror(int s) {
  switch (s) {
    case WDF_OK: return "success";
    case WDF_EINVAL: return "invalid argument";
    case WDF_ENOMEM: return "out of memory";
    case WDF_ECUDA: return "CUDA error";
    case WDF_ENOCONV: return "not converged";
    case WDF_ETIMEOUT: return "device wait timed out";
    case WDF_ENAN: return "non-finite value";
    case WDF_ESTATE: return "context or device unusable";
    default: return "unknown status";
  }
}

const char *wdf_last_error(const wdf_ctx *c) { return c ? c->err.c_str() : last_global_error(); }

const char *wdf_version(void) { return "wdf 0.1 (sm_103a)"; }

}  // extern "C"

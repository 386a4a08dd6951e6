// C ABI entry points of libwdf.so (declared in include/wdf.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>
#include <thread>
#include <algorithm>

#include "engine.cuh"

using namespace wdf;

namespace wdf {
static thread_local std::string g_last_error;
void set_error(int, const std::string &msg) { g_last_error = msg; }
const char *last_global_error() { return g_last_error.c_str(); }

thread_local Profiler *t_prof = nullptr;
std::atomic<long long> g_launches{0};

void raise_smem_limit_raw(const void *func, size_t bytes) {
  static std::mutex m;
  static std::map<std::pair<int, const void *>, size_t> cur;
  int dev = 0;
  WDF_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  size_t &c = cur[{dev, func}];
  if (bytes <= c) return;
  WDF_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  c = bytes;
}

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
  st->fallbacks = ss.fallbacks;
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
  c->miller.assign(sys->miller, sys->miller + 3 * (size_t)sys->npw_h);
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
  upload(c, c->t_jnat, L.jnat);
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
  g.ymax = L.ymax;
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
  c->f64.jnat = c->f32.jnat = c->fdf.jnat = c->t_jnat.as<int>();
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
  set_chol_inv_limits(kCholMax);
  set_mlp_limits();
  if (tc_enabled()) set_tc_limits();
  if (oz_enabled()) set_oz_limits();

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
    agg.fallbacks += ss.fallbacks;
    nsolve += (long long)n * c->nocc;
  }
};

// The caller's operator (wdf_davidson): internal vectors go out in the half-sphere layout to the
// callback and its results come back into the internal layout.
struct UserOp : DavOp {
  wdf_ctx *c;
  wdf_operator_fn fn;
  void *user;
  long long calls = 0;
  UserOp(wdf_ctx *cc, wdf_operator_fn f, void *u) : c(cc), fn(f), user(u) {}
  void apply(const cplx<double> *X, cplx<double> *Y, int n) override {
    const size_t nd = 2 * (size_t)n * c->npw_h;
    c->uop_in.ensure(nd * sizeof(double));
    c->uop_out.ensure(nd * sizeof(double));
    launch_int_to_ext(X, n, c->geo.ld, c->npw_h, c->t_emap.as<int>(), c->t_econj.as<int>(), c->uop_in.as<double>(), c->st);
    WDF_CUDA_TRY(cudaMemsetAsync(c->uop_out.p, 0, nd * sizeof(double), c->st));
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));  // the callback may work on any stream
    const int rc = fn(user, n, c->uop_in.as<double>(), c->uop_out.as<double>());
    if (rc != 0) throw ApiFailure(WDF_EINVAL, "the operator callback returned " + std::to_string(rc));
    ++calls;
    const size_t bytes = sizeof(cplx<double>) * (size_t)n * c->geo.ld;
    WDF_CUDA_TRY(cudaMemsetAsync(Y, 0, bytes, c->st));
    launch_ext_to_int(c->uop_out.as<double>(), n, c->npw_h, c->t_emap.as<int>(), c->t_emap2.as<int>(), c->t_econj.as<int>(), nullptr, Y,
                      c->geo.ld, c->st);
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
                  &c->flag,      &c->guess,     &c->chi_out, &c->chi_drho, &c->t_xactn, &c->t_jidx, &c->t_jnat,
                  &c->t_twdf,    &c->vlocdf,    &c->Udf,     &c->psirdf,   &c->dfa,     &c->dfb,
                  &c->xpdf,      &c->dvgriddf,  &c->accgriddf, &c->cb2df,  &c->drdf,    &c->oudf, &c->chol,
                  &c->ml64,      &c->ml32,      &c->mlw64,   &c->krow,     &c->rr_ref,  &c->it_ref,  &c->nfb,
                  &c->mlsums,    &c->mlwraw,    &c->tcU,     &c->tcUt,     &c->tcC,     &c->tcerr,
                  &c->wp_phi,    &c->wp_x,      &c->wp_y,    &c->wp_vx,    &c->wp_S,    &c->wp_coef,
                  &c->uop_in,    &c->uop_out,   &c->orbfields, &c->ones64,  &c->onesdf,  &c->pnorm,
                  &c->ozU,       &c->ozUe,      &c->ozUt,    &c->ozUte,    &c->ozPt,    &c->ozPte,   &c->ozX,
                  &c->ozXe,      &c->ozC,       &c->ozCe};
  for (DBuf *b : bufs) b->release();
  for (cudaEvent_t e : c->prof.ev) (void)cudaEventDestroy(e);
  for (wdf_ctx::Cg *w : {&c->cg64, &c->cg32, &c->cgdf}) {
    DBuf *cb[] = {&w->r,     &w->z,     &w->p,     &w->Ap, &w->x,  &w->cb, &w->S,  &w->part1,
                  &w->part2, &w->part3, &w->dbl, &w->ints, &w->r2, &w->p2, &w->cd, &w->ci, &w->cidx};
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

int wdf_set_residual_update(wdf_ctx *c, int on) {
  if (!c || (on != 0 && on != 1)) return WDF_EINVAL;
  c->opt.residual_update = on;
  return WDF_OK;
}

int wdf_apply_sternheimer_operator(wdf_ctx *c, int nvec, const int32_t *vidx, const double *in, double *out, int mem) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    check_mem(mem);
    if (nvec < 0 || (nvec > 0 && (!vidx || !in || !out))) throw ApiFailure(WDF_EINVAL, "bad nvec or NULL buffer");
    for (int s = 0; s < nvec; ++s)
      if (vidx[s] < 0 || vidx[s] >= c->nocc) throw ApiFailure(WDF_EINVAL, "vidx out of range");
    if (nvec == 0) return WDF_OK;
    cplx<double> *X = read_in(c, c->ext_in, c->xpert, in, nvec, mem);
    c->outi.ensure(sizeof(cplx<double>) * (size_t)nvec * c->geo.ld);
    std::vector<int> v(vidx, vidx + nvec);
    apply_sternheimer_operator(c, X, c->outi.as<cplx<double>>(), v.data(), nvec);
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

int wdf_apply_wp(wdf_ctx *c, int neig, const double *lambda, const double *phibar, int nvec, const double *in, double *out, int mem) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    check_mem(mem);
    if (neig < 1 || nvec < 0 || !lambda || !phibar || (nvec > 0 && (!in || !out))) throw ApiFailure(WDF_EINVAL, "bad arguments");
    std::vector<double> coef(neig);
    for (int a = 0; a < neig; ++a) {
      if (!(lambda[a] < 1.0)) throw ApiFailure(WDF_EINVAL, "an eigenvalue lambda >= 1 has no screening factor lambda / (1 - lambda)");
      coef[a] = lambda[a] / (1.0 - lambda[a]);
    }
    if (nvec == 0) return WDF_OK;
    cplx<double> *P = read_in(c, c->ext_in, c->wp_phi, phibar, neig, mem);
    cplx<double> *X = read_in(c, c->ext_out2, c->wp_x, in, nvec, mem);
    c->wp_coef.ensure(sizeof(double) * neig);
    WDF_CUDA_TRY(cudaMemcpyAsync(c->wp_coef.p, coef.data(), sizeof(double) * neig, cudaMemcpyHostToDevice, c->st));
    c->wp_y.ensure(sizeof(cplx<double>) * (size_t)nvec * c->geo.ld);
    wp_apply_internal(c, P, c->wp_coef.as<double>(), neig, X, nvec, c->wp_y.as<cplx<double>>());
    write_out(c, c->ext_out, c->wp_y.as<cplx<double>>(), nvec, out, mem);
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    return WDF_OK;
  });
}

int wdf_apply_chi0_multi(int nsys, wdf_ctx *const *ctx, const int *npert, const double *const *phi, double *const *out, int mem,
                         wdf_stats *st) {
  if (nsys < 1 || !ctx || !npert || !phi || !out) {
    set_error(WDF_EINVAL, "bad nsys or NULL array");
    return WDF_EINVAL;
  }
  for (int k = 0; k < nsys; ++k) {
    if (!ctx[k] || ctx[k]->device != ctx[0]->device) {
      set_error(WDF_EINVAL, "contexts must be non-NULL and on one GPU");
      return WDF_EINVAL;
    }
    for (int j = 0; j < k; ++j)
      if (ctx[j] == ctx[k]) {
        set_error(WDF_EINVAL, "a context appears twice");
        return WDF_EINVAL;
      }
  }
  // one host thread per system; a context on the legacy default stream gets a private stream
  // for the call so that the systems' kernels can overlap
  std::vector<int> rc(nsys, WDF_OK);
  std::vector<std::string> msg(nsys);
  auto work = [&](int k) {
    wdf_ctx *c = ctx[k];
    cudaStream_t saved = c->st, own = nullptr;
    if (!saved) {
      if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        rc[k] = WDF_ECUDA;
        msg[k] = "stream creation failed";
        return;
      }
      c->st = own;
    }
    rc[k] = wdf_apply_chi0(c, npert[k], phi[k], out[k], nullptr, mem, st ? &st[k] : nullptr);
    if (rc[k] != WDF_OK) msg[k] = c->err;
    if (own) {
      (void)cudaStreamSynchronize(own);
      (void)cudaStreamDestroy(own);
      c->st = saved;
    }
  };
  try {
    std::vector<std::thread> th;
    th.reserve(nsys);
    for (int k = 1; k < nsys; ++k) th.emplace_back(work, k);
    work(0);
    for (auto &t : th) t.join();
  } catch (const std::exception &) {
    set_error(WDF_EINVAL, "could not start the host threads");
    return WDF_EINVAL;
  }
  // the worst status wins: any error before not-converged
  int worst = WDF_OK;
  for (int k = 0; k < nsys; ++k) {
    if (rc[k] != WDF_OK && rc[k] != WDF_ENOCONV) {
      set_error(rc[k], "system " + std::to_string(k) + ": " + msg[k]);
      return rc[k];
    }
    if (rc[k] == WDF_ENOCONV) worst = WDF_ENOCONV;
  }
  return worst;
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

int wdf_davidson(wdf_ctx *c, wdf_operator_fn apply, void *user, int neig, int nbasis_max, int maxiter, double tol, int zero_g0,
                 int nguess, const double *guess, double *lambda, double *vec, int mem, wdf_stats *st) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    Timer tm;
    check_mem(mem);
    if (!apply || neig < 1 || nguess < neig || !guess || !lambda || !vec || maxiter < 1 || !(tol > 0) || nbasis_max < 0)
      throw ApiFailure(WDF_EINVAL, "bad Davidson arguments");
    const int dim = 2 * c->geo.nint - c->geo.len0 - (zero_g0 ? 1 : 0);
    if (neig > dim) throw ApiFailure(WDF_EINVAL, "neig exceeds the basis dimension");
    const int nbmax = nbasis_max > 0 ? nbasis_max : 4 * neig;
    cplx<double> *G0 = read_in(c, c->ext_in, c->guess, guess, nguess, mem);
    if (zero_g0) {
      const int e0 = c->lay.col_off[0] - c->lay.col_zlo[0];
      WDF_CUDA_TRY(cudaMemset2DAsync(G0 + e0, sizeof(cplx<double>) * c->geo.ld, 0, sizeof(cplx<double>), nguess, c->st));
    }
    UserOp op(c, apply, user);
    DavResult r = davidson(c, op, G0, nguess, neig, neig, nbmax, maxiter, tol, zero_g0 != 0);
    for (int a = 0; a < neig; ++a) lambda[a] = r.lam[a];
    write_out(c, c->ext_out, c->dv_X.as<cplx<double>>(), neig, vec, mem);
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    SolveStats none;
    none.converged = r.converged;
    fill_stats(st, none, 0, r.napply, tm.ms());
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
    c->prof.blocks = 0;
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

int wdf_profile_units(wdf_ctx *c, int64_t *blocks) {
  if (!c || !blocks) return WDF_EINVAL;
  *blocks = c->prof.blocks;
  return WDF_OK;
}

int wdf_plane_variant(const wdf_ctx *c, int bits, int *variant) {
  if (!c || !variant) return WDF_EINVAL;
  switch (bits) {
    case 32: *variant = c->f32.vloc_variant; return WDF_OK;
    case 64: *variant = c->opt.precision == WDF_MIXED_DF ? 0 : c->f64.vloc_variant; return WDF_OK;
    case 48: *variant = c->opt.precision == WDF_MIXED_DF ? c->fdf.vloc_variant : 0; return WDF_OK;
    default: return WDF_EINVAL;
  }
}

int64_t wdf_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t wdf_device_bytes(void) { return (int64_t)g_dev_bytes.load(); }

int64_t wdf_alloc_count(void) { return (int64_t)g_dev_allocs.load(); }

void wdf_set_device_limit(int64_t bytes) { g_dev_cap.store(bytes > 0 ? (long long)bytes : 0); }

int wdf_set_wait_limit(wdf_ctx *c, int64_t polls) {
  if (!c) return WDF_EINVAL;
  c->wait_polls = polls > 0 ? (long)polls : 0;
  return WDF_OK;
}

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

// ---------------------------------------------------------------------------------------------
// learned preconditioner models

namespace {

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): state += golden gamma, then the variant-13
// finaliser; output k of seed s is the finaliser of s + (k + 1) gamma
uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// uniform in (0, 1) from the top 53 bits
double unit_open(uint64_t x) { return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
// standard normal number k of a stream (Box-Muller on two consecutive outputs)
double normal_at(uint64_t seed, uint64_t k) {
  const double u1 = unit_open(splitmix64(seed, 2 * k)), u2 = unit_open(splitmix64(seed, 2 * k + 1));
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// n vectors of np half-sphere coefficients: Gaussian real and imaginary parts from
// splitmix64(seed) (entry pair k of vector p uses outputs 2 (p np + i), +1), G = 0 set to zero,
// each scaled to unit Gamma norm a0^2 + 2 sum_{G != 0} |a_G|^2
std::vector<double> gaussian_vectors(uint64_t seed, int n, int np) {
  std::vector<double> v(2 * (size_t)n * np);
  for (int p = 0; p < n; ++p) {
    double nrm = 0.0;
    for (int i = 0; i < np; ++i) {
      double *c2 = &v[2 * ((size_t)p * np + i)];
      const uint64_t idx = 2 * ((uint64_t)p * np + i);
      c2[0] = i == 0 ? 0.0 : normal_at(seed, idx);
      c2[1] = i == 0 ? 0.0 : normal_at(seed, idx + 1);
      nrm += 2.0 * (c2[0] * c2[0] + c2[1] * c2[1]);
    }
    const double sc = nrm > 0 ? 1.0 / std::sqrt(nrm) : 0.0;
    for (int i = 0; i < 2 * np; ++i) v[2 * (size_t)p * np + i] *= sc;
  }
  return v;
}

template <class F> int mguard(wdf_model *m, F &&body) {
  try {
    cudaError_t e = cudaSetDevice(m->device);
    if (e != cudaSuccess) throw CudaFailure(e, "cudaSetDevice", __FILE__, __LINE__);
    return body();
  } catch (const ApiFailure &f) {
    m->err = f.msg;
    set_error(f.code, f.msg);
    return f.code;
  } catch (const CudaFailure &f) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(f.err), cudaGetErrorString(f.err), f.what,
             f.file, f.line);
    m->err = buf;
    set_error(WDF_ECUDA, buf);
    return WDF_ECUDA;
  } catch (const std::bad_alloc &) {
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  } catch (...) {
    set_error(WDF_EINVAL, "unexpected C++ exception");
    return WDF_EINVAL;
  }
}

// grow a buffer keeping its first `used` bytes
void grow_keep(DBuf &b, size_t used, size_t need) {
  if (need <= b.cap) return;
  DBuf nb;
  nb.ensure(std::max(need, 2 * b.cap));
  if (used) WDF_CUDA_TRY(cudaMemcpy(nb.p, b.p, used, cudaMemcpyDeviceToDevice));
  b.release();
  b = nb;
}

void model_reserve(wdf_model *m, long long n) {
  if (n <= m->cap) return;
  const long long cap = std::max<long long>(n, 2 * m->cap);
  grow_keep(m->feat, sizeof(float) * 4 * m->n, sizeof(float) * 4 * cap);
  grow_keep(m->tgt, sizeof(float) * 2 * m->n, sizeof(float) * 2 * cap);
  grow_keep(m->wt, sizeof(float) * 2 * m->n, sizeof(float) * 2 * cap);
  m->cap = cap;
}

void model_upload(wdf_model *m, const std::vector<double> &w) {
  std::vector<float> f(w.begin(), w.end());
  WDF_CUDA_TRY(cudaMemcpy(m->w64.p, w.data(), sizeof(double) * kMlpFloats, cudaMemcpyHostToDevice));
  WDF_CUDA_TRY(cudaMemcpy(m->w32.p, f.data(), sizeof(float) * kMlpFloats, cudaMemcpyHostToDevice));
  WDF_CUDA_TRY(cudaMemset(m->m.p, 0, sizeof(double) * kMlpParams));
  WDF_CUDA_TRY(cudaMemset(m->v.p, 0, sizeof(double) * kMlpParams));
  m->t = 0;
}

// loss and gradient at the current weights into m->grad (device)
void model_grad(wdf_model *m) {
  set_mlp_limits();
  m->part.ensure(sizeof(double) * (kMlpParams + 1) * (size_t)mlp_grad_blocks(m->n));
  launch_mlp_grad(m->w32.as<float>(), m->feat.as<float>(), m->tgt.as<float>(), m->wt.as<float>(), m->n, m->part.as<double>(),
                  m->grad.as<double>(), 0);
}

}  // namespace

extern "C" {

void wdf_default_train_opts(wdf_train_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->steps = 600;
  o->lr = 3e-3;
  o->npert = 8;
  o->seed = 0;
}

int wdf_model_create(int device, uint64_t seed, wdf_model **out) {
  if (!out) {
    set_error(WDF_EINVAL, "out must not be NULL");
    return WDF_EINVAL;
  }
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    set_error(WDF_ESTATE, "no CUDA device available");
    return WDF_ESTATE;
  }
  if (device < 0 || device >= ndev) {
    set_error(WDF_EINVAL, "device ordinal out of range");
    return WDF_EINVAL;
  }
  wdf_model *m = new (std::nothrow) wdf_model();
  if (!m) {
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  }
  m->device = device;
  const int rc = mguard(m, [&] {
    m->w64.ensure(sizeof(double) * kMlpFloats);
    m->w32.ensure(sizeof(float) * kMlpFloats);
    m->m.ensure(sizeof(double) * kMlpParams);
    m->v.ensure(sizeof(double) * kMlpParams);
    m->grad.ensure(sizeof(double) * (kMlpParams + 1));
    // weights: normal with variance 1 / fan-in (4, 64, 64); biases 0; mu 0, sd 1
    std::vector<double> w(kMlpFloats, 0.0);
    const int fan_off[3][3] = {{0, 256, 4}, {320, 4096, 64}, {4480, 128, 64}};
    uint64_t k = 0;
    for (auto &L : fan_off)
      for (int i = 0; i < L[1]; ++i) w[L[0] + i] = normal_at(seed, k++) / std::sqrt((double)L[2]);
    for (int i = 0; i < 4; ++i) w[kMlpParams + 4 + i] = 1.0;
    model_upload(m, w);
    m->fresh = true;
    return WDF_OK;
  });
  if (rc != WDF_OK) {
    wdf_model_free(m);
    return rc;
  }
  *out = m;
  return WDF_OK;
}

void wdf_model_free(wdf_model *m) {
  if (!m) return;
  (void)cudaSetDevice(m->device);
  (void)cudaDeviceSynchronize();
  for (DBuf *b : {&m->w64, &m->w32, &m->m, &m->v, &m->grad, &m->part, &m->feat, &m->tgt, &m->wt, &m->pin, &m->pout}) b->release();
  delete m;
}

int wdf_model_set_weights(wdf_model *m, const float *w) {
  if (!m || !w) return WDF_EINVAL;
  return mguard(m, [&] {
    std::vector<double> d(w, w + kMlpFloats);
    for (int i = 0; i < 4; ++i)
      if (!(d[kMlpParams + 4 + i] > 0)) throw ApiFailure(WDF_EINVAL, "sd entries must be positive");
    for (double x : d)
      if (!std::isfinite(x)) throw ApiFailure(WDF_ENAN, "non-finite weight");
    model_upload(m, d);
    m->fresh = false;
    return WDF_OK;
  });
}

int wdf_model_get_weights(const wdf_model *mc, float *w) {
  wdf_model *m = const_cast<wdf_model *>(mc);
  if (!m || !w) return WDF_EINVAL;
  return mguard(m, [&] {
    WDF_CUDA_TRY(cudaMemcpy(w, m->w32.p, sizeof(float) * kMlpFloats, cudaMemcpyDeviceToHost));
    return WDF_OK;
  });
}

int64_t wdf_model_num_samples(const wdf_model *m) { return m ? (int64_t)m->n : -1; }

int wdf_model_set_samples(wdf_model *m, int64_t n, const float *feat, const float *tgt, const float *wt) {
  if (!m || n < 0 || (n > 0 && (!feat || !tgt || !wt))) return WDF_EINVAL;
  return mguard(m, [&] {
    m->n = 0;
    model_reserve(m, n);
    if (n > 0) {
      WDF_CUDA_TRY(cudaMemcpy(m->feat.p, feat, sizeof(float) * 4 * n, cudaMemcpyHostToDevice));
      WDF_CUDA_TRY(cudaMemcpy(m->tgt.p, tgt, sizeof(float) * 2 * n, cudaMemcpyHostToDevice));
      WDF_CUDA_TRY(cudaMemcpy(m->wt.p, wt, sizeof(float) * 2 * n, cudaMemcpyHostToDevice));
    }
    m->n = n;
    return WDF_OK;
  });
}

int wdf_model_get_samples(const wdf_model *mc, int64_t first, int64_t count, float *feat, float *tgt, float *wt) {
  wdf_model *m = const_cast<wdf_model *>(mc);
  if (!m || first < 0 || count < 0 || first + count > m->n) return WDF_EINVAL;
  return mguard(m, [&] {
    if (count == 0) return WDF_OK;
    if (feat) WDF_CUDA_TRY(cudaMemcpy(feat, m->feat.as<float>() + 4 * first, sizeof(float) * 4 * count, cudaMemcpyDeviceToHost));
    if (tgt) WDF_CUDA_TRY(cudaMemcpy(tgt, m->tgt.as<float>() + 2 * first, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost));
    if (wt) WDF_CUDA_TRY(cudaMemcpy(wt, m->wt.as<float>() + 2 * first, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost));
    return WDF_OK;
  });
}

int wdf_model_add_solves(wdf_model *m, wdf_ctx *c, int npert, const double *phi, int mem, wdf_stats *st) {
  if (!m || !c) return WDF_EINVAL;
  if (m->device != c->device) {
    set_error(WDF_EINVAL, "the model and the context live on different GPUs");
    return WDF_EINVAL;
  }
  return guarded(c, [&] {
    Timer tm;
    check_mem(mem);
    if (npert < 1 || !phi) throw ApiFailure(WDF_EINVAL, "bad npert or NULL phi");
    const Geo &g = c->geo;
    cplx<double> *P = read_in(c, c->ext_in, c->guess, phi, npert, mem, 1);
    const int np2 = 2 * ((npert + 1) / 2);
    c->outi.ensure(sizeof(cplx<double>) * (size_t)np2 * g.ld);
    c->drhoi.ensure(sizeof(cplx<double>) * (size_t)np2 * g.ld);
    c->mlsums.ensure(sizeof(double) * 3 * (size_t)c->nocc * g.ld);
    WDF_CUDA_TRY(cudaMemsetAsync(c->mlsums.p, 0, sizeof(double) * 3 * (size_t)c->nocc * g.ld, c->st));
    // TPA solves with the sums collected; the options come back whatever happens
    struct Restore {
      wdf_ctx *c;
      int precond;
      ~Restore() {
        c->opt.precond = precond;
        c->collect = false;
      }
    } restore{c, c->opt.precond};
    c->opt.precond = WDF_PRECOND_TPA;
    c->collect = true;
    SolveStats ss;
    chi0_apply_internal(c, P, npert, c->outi.as<cplx<double>>(), c->drhoi.as<cplx<double>>(), ss);
    const long long add = (long long)c->nocc * c->npw_h;
    model_reserve(m, m->n + add);
    c->mlwraw.ensure(sizeof(double) * (2 * (size_t)add + 2));
    double *wraw = c->mlwraw.as<double>();
    launch_mlp_samples(g, c->t_emap.as<int>(), c->npw_h, c->nocc, c->mlsums.as<double>(),
                       c->U64.as<cplx<double>>() + (size_t)c->nproj * g.ld, c->tkin.as<double>(), c->eps_dev.as<double>(),
                       m->feat.as<float>() + 4 * m->n, m->tgt.as<float>() + 2 * m->n, m->wt.as<float>() + 2 * m->n, wraw,
                       wraw + 2 * add, c->st);
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    m->n += add;
    fill_stats(st, ss, (long long)npert * c->nocc, npert, tm.ms());
    return ss.converged ? WDF_OK : WDF_ENOCONV;
  });
}

int wdf_model_loss_grad(wdf_model *m, double *loss, double *grad) {
  if (!m || !loss || !grad) return WDF_EINVAL;
  return mguard(m, [&] {
    if (m->n == 0) throw ApiFailure(WDF_EINVAL, "the model has no samples");
    model_grad(m);
    std::vector<double> h(kMlpParams + 1);
    WDF_CUDA_TRY(cudaMemcpy(h.data(), m->grad.p, sizeof(double) * (kMlpParams + 1), cudaMemcpyDeviceToHost));
    std::copy(h.begin(), h.begin() + kMlpParams, grad);
    *loss = h[kMlpParams];
    return WDF_OK;
  });
}

int wdf_model_train(wdf_model *m, const wdf_train_opts *opt, wdf_train_stats *st) {
  if (!m) return WDF_EINVAL;
  wdf_train_opts o;
  if (opt) o = *opt;
  else wdf_default_train_opts(&o);
  return mguard(m, [&] {
    auto t0 = std::chrono::steady_clock::now();
    if (m->n == 0) throw ApiFailure(WDF_EINVAL, "the model has no samples");
    if (o.steps < 0 || !(o.lr > 0)) throw ApiFailure(WDF_EINVAL, "bad training options");
    if (m->fresh && m->t == 0) {
      // feature normalisation and output biases from the samples (host, FP64)
      const long long n = m->n;
      std::vector<float> f(4 * n), t(2 * n), w(2 * n);
      WDF_CUDA_TRY(cudaMemcpy(f.data(), m->feat.p, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost));
      WDF_CUDA_TRY(cudaMemcpy(t.data(), m->tgt.p, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost));
      WDF_CUDA_TRY(cudaMemcpy(w.data(), m->wt.p, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost));
      std::vector<double> wd(kMlpFloats);
      WDF_CUDA_TRY(cudaMemcpy(wd.data(), m->w64.p, sizeof(double) * kMlpFloats, cudaMemcpyDeviceToHost));
      for (int k = 0; k < 4; ++k) {
        double s1 = 0.0, s2 = 0.0;
        for (long long i = 0; i < n; ++i) s1 += f[4 * i + k];
        const double mu = s1 / (double)n;
        for (long long i = 0; i < n; ++i) s2 += (f[4 * i + k] - mu) * (f[4 * i + k] - mu);
        const double sd = std::sqrt(s2 / (double)n);
        wd[kMlpParams + k] = mu;
        wd[kMlpParams + 4 + k] = sd > 1e-6 ? sd : 1.0;
      }
      for (int k = 0; k < 2; ++k) {
        double sw = 0.0, st2 = 0.0;
        for (long long i = 0; i < n; ++i) {
          sw += w[2 * i + k];
          st2 += (double)w[2 * i + k] * t[2 * i + k];
        }
        wd[kMlpParams - 2 + k] = sw > 0 ? st2 / sw : 0.0;
      }
      model_upload(m, wd);
    }
    double first = 0.0, last = 0.0;
    for (int s = 0; s < o.steps; ++s) {
      model_grad(m);
      if (s == 0 || s == o.steps - 1) {
        double l = 0.0;
        WDF_CUDA_TRY(cudaMemcpy(&l, m->grad.as<double>() + kMlpParams, sizeof(double), cudaMemcpyDeviceToHost));
        if (!std::isfinite(l)) throw ApiFailure(WDF_ENAN, "non-finite training loss");
        if (s == 0) first = l;
        last = l;
      }
      launch_mlp_adam(m->w64.as<double>(), m->w32.as<float>(), m->grad.as<double>(), m->m.as<double>(), m->v.as<double>(), ++m->t,
                      o.lr, 0);
    }
    WDF_CUDA_TRY(cudaDeviceSynchronize());
    m->fresh = false;
    if (st) {
      st->nsamples = m->n;
      st->steps = o.steps;
      st->loss_first = first;
      st->loss_last = last;
      st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return WDF_OK;
  });
}

int wdf_model_predict(wdf_model *m, int64_t n, const float *feat, float *out) {
  if (!m || n < 0 || (n > 0 && (!feat || !out))) return WDF_EINVAL;
  return mguard(m, [&] {
    if (n == 0) return WDF_OK;
    m->pin.ensure(sizeof(float) * 4 * n);
    m->pout.ensure(sizeof(float) * 2 * n);
    WDF_CUDA_TRY(cudaMemcpy(m->pin.p, feat, sizeof(float) * 4 * n, cudaMemcpyHostToDevice));
    launch_mlp_predict(m->w32.as<float>(), m->pin.as<float>(), n, m->pout.as<float>(), 0);
    WDF_CUDA_TRY(cudaMemcpy(out, m->pout.p, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost));
    return WDF_OK;
  });
}

int wdf_set_model(wdf_ctx *c, const wdf_model *m) {
  if (!c) return WDF_EINVAL;
  return guarded(c, [&] {
    if (!m) {
      c->opt.precond = WDF_PRECOND_TPA;
      c->has_model = false;
      return WDF_OK;
    }
    if (m->device != c->device) throw ApiFailure(WDF_EINVAL, "the model and the context live on different GPUs");
    // the model's weights were written on the default stream: order them before the table
    WDF_CUDA_TRY(cudaDeviceSynchronize());
    const Geo &g = c->geo;
    const size_t rows = 2 * (size_t)c->nocc * g.ld;
    c->ml64.ensure(sizeof(double) * rows);
    c->ml32.ensure(sizeof(float) * rows);
    c->mlw64.ensure(sizeof(double) * (size_t)c->nocc * g.ld);
    launch_mlp_table(g, m->w32.as<float>(), c->U64.as<cplx<double>>() + (size_t)c->nproj * g.ld, c->tkin.as<double>(),
                     c->eps_dev.as<double>(), c->npw_h, c->kp64.as<double>(), c->nocc, c->ml64.as<double>(), c->ml32.as<float>(),
                     c->mlw64.as<double>(), c->st);
    int bad = 0;
    c->flag.ensure(sizeof(int));
    WDF_CUDA_TRY(cudaMemsetAsync(c->flag.p, 0, sizeof(int), c->st));
    launch_check_finite<double>(c->ml64.as<double>(), rows, c->flag.as<int>(), c->st);
    WDF_CUDA_TRY(cudaMemcpyAsync(&bad, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WDF_CUDA_TRY(cudaStreamSynchronize(c->st));
    if (bad) throw ApiFailure(WDF_ENAN, "the model gives non-finite preconditioner values");
    c->opt.precond = WDF_PRECOND_LEARNED;
    c->has_model = true;
    return WDF_OK;
  });
}

int wdf_train_preconditioner(wdf_ctx *const *ctx, int n, const wdf_train_opts *opt, wdf_model **out, wdf_train_stats *st) {
  if (!out) return WDF_EINVAL;
  *out = nullptr;
  if (!ctx || n < 1) return WDF_EINVAL;
  for (int k = 0; k < n; ++k)
    if (!ctx[k] || ctx[k]->device != ctx[0]->device) {
      set_error(WDF_EINVAL, "contexts must be non-NULL and on one GPU");
      return WDF_EINVAL;
    }
  wdf_train_opts o;
  if (opt) o = *opt;
  else wdf_default_train_opts(&o);
  if (o.npert < 1) return WDF_EINVAL;
  wdf_model *m = nullptr;
  int rc = wdf_model_create(ctx[0]->device, o.seed, &m);
  if (rc != WDF_OK) return rc;
  for (int k = 0; k < n && rc == WDF_OK; ++k) {
    // perturbations: Gaussian coefficients from splitmix64(seed + k + 1), G = 0 removed, unit norm
    const std::vector<double> phi = gaussian_vectors(o.seed + (uint64_t)k + 1, o.npert, ctx[k]->npw_h);
    rc = wdf_model_add_solves(m, ctx[k], o.npert, phi.data(), WDF_MEM_HOST, nullptr);
    if (rc == WDF_ENOCONV) rc = WDF_OK;  // samples of unconverged solves are still usable
  }
  if (rc == WDF_OK) rc = wdf_model_train(m, &o, st);
  if (rc != WDF_OK) {
    wdf_model_free(m);
    return rc;
  }
  *out = m;
  return WDF_OK;
}


int wdf_half_sphere(const double cell[9], double ecut, int32_t *miller, int *npw_h) {
  if (!cell || !npw_h || !(ecut > 0)) {
    set_error(WDF_EINVAL, "cell, npw_h and a positive ecut are required");
    return WDF_EINVAL;
  }
  try {
    const double *A = cell;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 0)) throw ApiFailure(WDF_EINVAL, "singular cell");
    // reciprocal rows b_i = 2 pi (A^-1)^T rows; |n_a| <= sqrt(ecut) |a_a| / (2 pi) bounds the box
    double B[9];
    const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det, (A[1] * A[5] - A[2] * A[4]) / det,
                           (A[5] * A[6] - A[3] * A[8]) / det, (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                           (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det, (A[0] * A[4] - A[1] * A[3]) / det};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
    int nm[3];
    for (int a = 0; a < 3; ++a) {
      const double la = std::sqrt(A[3 * a] * A[3 * a] + A[3 * a + 1] * A[3 * a + 1] + A[3 * a + 2] * A[3 * a + 2]);
      nm[a] = (int)std::floor(std::sqrt(ecut) * la / (2.0 * M_PI) + 1e-9);
      if (nm[a] > 4096) throw ApiFailure(WDF_EINVAL, "cutoff too large for the cell");
    }
    struct Gv {
      long long key;
      int n1, n2, n3;
    };
    std::vector<Gv> gv;
    for (int n3 = 0; n3 <= nm[2]; ++n3)
      for (int n2 = (n3 > 0 ? -nm[1] : 0); n2 <= nm[1]; ++n2)
        for (int n1 = ((n3 > 0 || n2 > 0) ? -nm[0] : 0); n1 <= nm[0]; ++n1) {
          double g[3];
          for (int c2 = 0; c2 < 3; ++c2) g[c2] = n1 * B[c2] + n2 * B[3 + c2] + n3 * B[6 + c2];
          const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          if (g2 > ecut * (1.0 + 1e-12)) continue;
          gv.push_back({std::llround(g2 * 1e9 / ecut), n1, n2, n3});  // shells binned at 1e-9 ecut
        }
    std::sort(gv.begin(), gv.end(), [](const Gv &a, const Gv &b) {
      if (a.key != b.key) return a.key < b.key;
      if (a.n1 != b.n1) return a.n1 < b.n1;
      if (a.n2 != b.n2) return a.n2 < b.n2;
      return a.n3 < b.n3;
    });
    if (miller) {
      if (*npw_h < (int)gv.size()) throw ApiFailure(WDF_EINVAL, "miller has room for fewer triples than the sphere holds");
      for (size_t i = 0; i < gv.size(); ++i) {
        miller[3 * i] = gv[i].n1;
        miller[3 * i + 1] = gv[i].n2;
        miller[3 * i + 2] = gv[i].n3;
      }
    }
    *npw_h = (int)gv.size();
    return WDF_OK;
  } catch (const ApiFailure &f) {
    set_error(f.code, f.msg);
    return f.code;
  } catch (...) {
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  }
}

int wdf_get_gvectors(const wdf_ctx *c, int32_t *miller) {
  if (!c || !miller) return WDF_EINVAL;
  std::copy(c->miller.begin(), c->miller.end(), miller);
  return WDF_OK;
}

int wdf_reset_error(wdf_ctx *c) {
  if (!c) return WDF_EINVAL;
  if (!c->failed) return WDF_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return WDF_ESTATE;
  (void)cudaGetLastError();  // a refused launch leaves a non-sticky error behind
  const cudaError_t e = c->st ? cudaStreamSynchronize(c->st) : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    c->err = std::string("the device reports ") + cudaGetErrorName(e) + ": the context stays unusable";
    return WDF_ESTATE;
  }
  if (c->tcerr.p && cudaMemset(c->tcerr.p, 0, sizeof(int)) != cudaSuccess) return WDF_ESTATE;  // bounded-wait flag
  c->failed = false;
  c->err.clear();
  return WDF_OK;
}

int wdf_pdep_davidson_seeded(wdf_ctx *c, int neig, int nbasis_max, int maxiter, double tol, uint64_t seed, double *lambda,
                             double *phibar, int mem, wdf_stats *st) {
  if (!c || neig < 1) return WDF_EINVAL;
  std::vector<double> guess;
  try {
    guess = gaussian_vectors(seed, neig, c->npw_h);
  } catch (...) {
    set_error(WDF_ENOMEM, "host allocation failed");
    return WDF_ENOMEM;
  }
  if (mem != WDF_MEM_DEVICE) return wdf_pdep_davidson(c, neig, nbasis_max, maxiter, tol, neig, guess.data(), lambda, phibar, mem, st);
  // device outputs: the start block goes to the device first
  DBuf dg;
  int rc = guarded(c, [&] {
    dg.ensure(sizeof(double) * guess.size());
    WDF_CUDA_TRY(cudaMemcpy(dg.p, guess.data(), sizeof(double) * guess.size(), cudaMemcpyHostToDevice));
    return WDF_OK;
  });
  if (rc == WDF_OK) rc = wdf_pdep_davidson(c, neig, nbasis_max, maxiter, tol, neig, dg.as<double>(), lambda, phibar, mem, st);
  (void)cudaSetDevice(c->device);
  dg.release();
  return rc;
}

}  // extern "C"

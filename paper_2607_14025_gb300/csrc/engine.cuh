// Host-side engine of libwdf.so: the context, its device buffers and the solver entry points.
#pragma once

#include <string>
#include <vector>

#include "kernels.cuh"

namespace wdf {

// Grow-only device buffer. ensure() may reallocate (contents are not kept).
struct DBuf {
  void *p = nullptr;
  size_t cap = 0;
  template <class T> T *as() const { return static_cast<T *>(p); }
  void ensure(size_t bytes);
  void release();
};
// device bytes held by all DBufs of the process, cudaMalloc calls made for them, and the cap
// on the bytes held (0: none); see layout.cu
extern std::atomic<long long> g_dev_bytes, g_dev_allocs, g_dev_cap;

// Host copy of the plane-wave layout (see layout.cu for its construction).
struct Layout {
  int K = 0, ndisk = 0, nint = 0, ld = 0, len0 = 0, ldcb = 0;
  std::vector<int> col_n1, col_n2, col_zlo, col_off;
  std::vector<int> e_col, e_z;
  std::vector<double> g2, vhalf;
  std::vector<int> tile_idx, xact, xactn, jidx, jnat;  // jnat: natural y * n1 + x of each disk column
  int xmax = 0;
  int ymax = 0;
  std::vector<short> pos3;
  std::vector<int> emap, emap2, econj;  // external half-sphere index -> internal element
  Plan1D P1, P2, P3;
};

// Build the layout; throws ApiFailure(WDF_EINVAL) on an invalid Miller set.
Layout build_layout(const int32_t *miller, int npw_h, const int n[3], const double bvec[9]);
Plan1D make_plan(int n);
std::vector<int> digit_reversal(const Plan1D &P);

}  // namespace wdf

struct wdf_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  wdf_options opt{};
  std::string err;
  bool failed = false;
  long wait_polls = 0;  // wdf_set_wait_limit: polls of software device waits (0: the default)

  // system
  int n[3] = {0, 0, 0};
  size_t ngrid = 0;
  double cell[9] = {0}, bvec[9] = {0}, omega = 0;
  int npw_h = 0, nproj = 0, nocc = 0;
  std::vector<double> dij, eps;
  std::vector<int32_t> miller;  // [npw_h][3] as given at setup
  double alpha = 0;
  double gap = 0;  // eps_{nocc+1} - eps_nocc when the library computed the ground state (else 0)

  wdf::Layout lay;
  wdf::Geo geo{};
  wdf::FftCtx<double> f64{};
  wdf::FftCtx<float> f32{};
  wdf::FftCtx<wdf::df64> fdf{};  // double-float instances (WDF_MIXED_DF)

  // layout tables
  wdf::DBuf t_col_off, t_col_zlo, t_e_col, t_e_z, t_tile, t_xact, t_pos3, t_g2, t_vhalf;
  wdf::DBuf t_emap, t_emap2, t_econj, t_tw64, t_tw32, t_twdf, t_xactn, t_jidx, t_jnat;

  // operator data
  wdf::DBuf vloc64, vloc32;  // V_loc on the grid
  wdf::DBuf U64, U32;        // [nproj + nocc][ld]: projectors then occupied orbitals (internal layout)
  wdf::DBuf lrd;             // [nproj + nocc]: D_j then alpha
  wdf::DBuf psir64, psir32;  // [nocc][ngrid] psi_v(r) (unnormalised inverse transform)
  wdf::DBuf kp64, kp32;      // [nocc][ld] TPA preconditioner
  wdf::DBuf tkin;            // [nocc]
  wdf::DBuf vlocdf, Udf, psirdf;  // double-float copies (WDF_MIXED_DF)
  wdf::DBuf eps_dev;         // [nocc]

  // workspaces (grow-only)
  struct Cg {
    wdf::DBuf r, z, p, Ap, x, cb, S, part1, part2, part3, dbl, ints;
    wdf::DBuf r2, p2, cd, ci, cidx;  // compacted copies of the active solves' rows and state
  } cg64, cg32, cgdf;
  // learned preconditioner (wdf_set_model): [2 nocc][ld] tables (learned rows, then TPA rows),
  // first-iterate gains [nocc][ld]; per-solve row index, stall-check state and fallback counter
  wdf::DBuf ml64, ml32, mlw64, krow, rr_ref, it_ref, nfb;
  // tensor-core projections of the FP32 CG: weighted U (hi, lo) [M][2 ld], U^T (hi, lo)
  // [2 ld][kp], coefficient staging, wait-expiry flag
  wdf::DBuf tcU, tcUt, tcC, tcerr;
  bool tc_on = false;
  float *tc_uwh() const { return tcU.as<float>(); }
  float *tc_uwl() const { return tcU.as<float>() + (size_t)(nproj + nocc) * 2 * geo.ld; }
  float *tc_uth() const { return tcUt.as<float>(); }
  float *tc_utl() const { return tcUt.as<float>() + (size_t)2 * geo.ld * wdf::tc_rows(nproj + nocc); }
  // tensor-core double-float projections (exact integer digits): digits of the weighted rows of
  // U, of U^T (all rows) and of psi^T (the orbital rows), and their exponents; workspaces for
  // the digits of the vectors and of the coefficients
  wdf::DBuf ozU, ozUe, ozUt, ozUte, ozPt, ozPte, ozX, ozXe, ozC, ozCe;
  wdf::OzMat oz_u, oz_ut, oz_pt;
  bool oz_on = false;
  bool has_model = false;
  // training-sample collection (wdf_model_add_solves): sums [3][nocc][ld] over converged solves
  wdf::DBuf mlsums, mlwraw;
  wdf::DBuf wp_phi, wp_x, wp_y, wp_vx, wp_S, wp_coef;  // wdf_apply_wp
  wdf::DBuf uop_in, uop_out;                           // wdf_davidson: the caller's operator's in / out
  wdf::DBuf pnorm;                      // squared norms of a block's perturbations
  wdf::DBuf orbfields, ones64, onesdf;  // orbital sum by G2R: one pair's real-space fields per orbital; psi = 1 grids
  bool collect = false;
  wdf::DBuf rb, rx, rr, rAx, rwork;        // refinement: b, x, r, A x (FP64), FP32 staging
  wdf::DBuf shift, vidx_dev, thr;          // per-solve shift, orbital index, thresholds
  wdf::DBuf gramw;                         // split partial sums of Gram products
  wdf::DBuf xpert, dvgrid, accgrid, cb2, outi, drhoi, ext_in, ext_out, ext_out2;
  wdf::DBuf dv_V, dv_W, dv_X, dv_AX, dv_R, dv_H, dv_Y, dv_theta, dv_jac, dv_jint, dv_small, dv_neg;
  wdf::DBuf zeros, flag, guess, chi_out, chi_drho, chol;
  wdf::DBuf dfa, dfb, xpdf, dvgriddf, accgriddf, cb2df, drdf, oudf;  // double-float work

  // kernel timing (wdf_profile_kernel)
  wdf::Profiler prof;
  bool prof_on = false;
};

namespace wdf {

// operators (engine.cu)
template <typename T>
void apply_operator(wdf_ctx *c, const cplx<T> *X, cplx<T> *Y, int n, const double *shift, bool with_alpha);
// A_v x = (H - eps_v + alpha P) x in the precision of the residuals (FP64, or double-float for
// WDF_MIXED_DF); vidx_host: [n] orbital of each vector
void apply_sternheimer_operator(wdf_ctx *c, const cplx<double> *X, cplx<double> *Y, const int *vidx_host, int n);

struct SolveStats {
  long long iters = 0;
  int iters_max = 0;
  int refinements = 0;
  double max_res = 0;
  bool converged = true;
  int fallbacks = 0;  // learned preconditioner: solves that restarted with TPA
};

// Solve (H - eps_v + alpha P) x = b for n right-hand sides in internal FP64 layout.
void sternheimer_solve(wdf_ctx *c, const cplx<double> *b, cplx<double> *x, const int *vidx_host, int n, SolveStats &ss);

// chi0bar applied to npert internal vectors phi (FP64, internal layout); out and drho internal.
void chi0_apply_internal(wdf_ctx *c, const cplx<double> *phi, int npert, cplx<double> *out, cplx<double> *drho,
                         SolveStats &ss);

// generic block Davidson over internal FP64 vectors
struct DavOp {
  virtual ~DavOp() {}
  virtual void apply(const cplx<double> *X, cplx<double> *Y, int n) = 0;
  virtual bool precondition() const { return false; }
};
struct DavResult {
  std::vector<double> lam;
  std::vector<double> resnorm;
  int iters = 0;
  long long napply = 0;
  bool converged = false;
};
// V0: n0 start vectors (internal layout, device). nwant lowest must converge; nkeep Ritz pairs
// are carried (nkeep >= nwant). Output Ritz vectors (nkeep) are left in c->dv_X.
DavResult davidson(wdf_ctx *c, DavOp &op, const cplx<double> *V0, int n0, int nwant, int nkeep, int nbmax,
                   int maxiter, double tol, bool zero_g0);

// x[s] = w[v_s] b[s] elementwise (first iterate of a solve from a per-(v, e) gain table)
void launch_first_iterate(const Geo &g, cplx<double> *x, const cplx<double> *b, const double *w, const int *vidx, int n,
                          cudaStream_t st);

// W_p x = v^1/2 sum_a phibar_a coef_a <phibar_a, v^1/2 x>, coef_a = lambda_a / (1 - lambda_a)
// (device array), internal FP64 vectors
void wp_apply_internal(wdf_ctx *c, const cplx<double> *phib, const double *coef, int neig, const cplx<double> *x, int nvec,
                       cplx<double> *y);

void ground_state(wdf_ctx *c);     // fills U64 psi rows and c->eps
void finish_setup(wdf_ctx *c);     // derived tables once psi and eps are known

}  // namespace wdf

// A learned-preconditioner model on one GPU (include/wdf.h).
struct wdf_model {
  int device = 0;
  std::string err;
  wdf::DBuf w64, w32;          // weights: FP64 master copy (kMlpFloats), FP32 copy for the kernels
  wdf::DBuf m, v;              // Adam moments (kMlpParams doubles each)
  wdf::DBuf grad, part;        // gradient + loss (kMlpParams + 1), per-block partials
  wdf::DBuf feat, tgt, wt;     // samples: [cap][4], [cap][2], [cap][2] floats
  wdf::DBuf pin, pout;         // staging of wdf_model_predict
  long long n = 0, cap = 0;    // samples held, capacity
  int t = 0;                   // Adam steps taken
  bool fresh = true;           // weights from wdf_model_create: first training sets mu, sd, b3
};

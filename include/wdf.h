/*
 * wdf.h -- C ABI of the GB300 DFPT screening library (libwdf.so).
 *
 * The library applies the symmetrised independent-particle response
 *     chi0bar = v^1/2 chi0 v^1/2
 * to blocks of plane-wave perturbations by density-functional perturbation theory, and finds the
 * lowest eigenpairs of chi0bar by block Davidson (projective dielectric eigendecomposition,
 * PDEP). Paper: "The WEST code for large-scale excited-state materials simulations", Sec. 2.1
 * (W_p = v^1/2 chibar v^1/2; chibar from the PDEP eigenpairs of chi0bar, Eq. (5); the density
 * response from Sternheimer equations without empty states) and Sec. 3.3 (one Davidson solver).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: hartree atomic units (energies in hartree, lengths in bohr).
 * Plane waves: orthonormal b_G(r) = Omega^-1/2 exp(iG.r), Gamma point, real functions, so only
 *   the half sphere is stored: npw_h Miller triples with G = 0 first and, for every other G in
 *   the list, -G absent from it. A half-sphere vector is npw_h complex numbers stored as
 *   interleaved doubles (re, im), 2*npw_h doubles; a block of n vectors is n consecutive vectors.
 *   Inner product of two such vectors: a0 b0 + 2 Re sum_{G != 0} conj(a_G) b_G.
 * Real-space grids: n1*n2*n3 doubles, index i1 + n1*(i2 + n2*i3) for the point
 *   r = (i1/n1) a1 + (i2/n2) a2 + (i3/n3) a3.
 * Memory: arguments documented as "host or device" are read from host memory when the call's
 *   mem argument is WDF_MEM_HOST and from device memory of the context's GPU when it is
 *   WDF_MEM_DEVICE. Other pointers are always host memory. The library copies what it needs,
 *   never frees caller memory and keeps no caller pointer after a call returns.
 * Streams: all GPU work of a context runs on the stream given at setup (0: the legacy default
 *   stream). Calls return after their results are in the caller's buffer unless stated.
 * Errors: every int-returning call returns WDF_OK (0) or one of the codes below and never aborts
 *   the process; the GPU never traps. wdf_last_error() gives a message for the last failure.
 *   A CUDA failure inside a context marks it failed (WDF_ESTATE on later calls) until destroyed.
 */
#ifndef WDF_H
#define WDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum wdf_status {
  WDF_OK = 0,
  WDF_EINVAL = 1,   /* invalid argument or descriptor */
  WDF_ENOMEM = 2,   /* device or host allocation failed */
  WDF_ECUDA = 3,    /* CUDA runtime error (message in wdf_last_error) */
  WDF_ENOCONV = 4,  /* an iteration hit its limit; outputs hold the last iterate, stats filled */
  WDF_ETIMEOUT = 5, /* a bounded device-side wait expired (the context stays usable) */
  WDF_ENAN = 6,     /* non-finite value in an input or an iterate */
  WDF_ESTATE = 7    /* context unusable after an earlier CUDA failure, or no GPU */
};

enum wdf_mem { WDF_MEM_HOST = 0, WDF_MEM_DEVICE = 1 };

/* Arithmetic of the Sternheimer solves.
 * WDF_FP64: every FFT, product, projection and CG update in FP64.
 * WDF_MIXED: inner conjugate-gradient iterations in FP32 (FFTs, H application, projections);
 *   the residual b - A x, the accumulated solution, the right-hand sides, the density response
 *   and the Davidson linear algebra in FP64 (iterative refinement), so the stopping test is an
 *   FP64 residual.
 * WDF_MIXED_DF: as WDF_MIXED, but the FFTs and projections of the residuals, right-hand sides and
 *   density response run in double-float arithmetic (pairs of FP32 numbers, about 48 significant
 *   bits, relative error near 1e-14) on the FP32 units; vectors, sums and the Davidson algebra
 *   stay FP64. GB300 issues FP32 about 60 times faster than FP64. */
enum wdf_precision { WDF_FP64 = 0, WDF_MIXED = 1, WDF_MIXED_DF = 2 };

/* Preconditioner of the Sternheimer CG. WDF_PRECOND_TPA: Teter-Payne-Allan, K(x) with
 * x = (1/2 |G|^2) / T_v. WDF_PRECOND_LEARNED: s(v, G) K, s from a trained model (wdf_set_model);
 * a solve whose residual norm falls by less than 10% over 5 iterations restarts with TPA. */
enum wdf_precond { WDF_PRECOND_NONE = 0, WDF_PRECOND_TPA = 1, WDF_PRECOND_LEARNED = 2 };

typedef struct wdf_ctx wdf_ctx;

/* The model system. Paper Sec. 2.1, Eq. (1): H psi_i = eps_i psi_i with
 * H = -1/2 nabla^2 + V_loc(r) + sum_j |beta_j> D_j <beta_j| (local plus Kleinman-Bylander). */
typedef struct wdf_system {
  double cell[9];        /* lattice vectors a1, a2, a3 as rows (bohr); host */
  int n[3];              /* FFT grid n1, n2, n3; each a product of 2, 3, 5, at most 128 (FP64: 96) */
  int npw_h;             /* number of half-sphere plane waves */
  const int32_t *miller; /* [npw_h][3] Miller indices (host); G = 0 first; for each (n1, n2)
                            column the n3 values must form one interval over the full sphere */
  const double *vloc_r;  /* [n3][n2][n1] local potential on the grid (host or device) */
  int nproj;             /* number of projectors (may be 0) */
  const double *beta;    /* [nproj][npw_h] complex projector coefficients (host or device) */
  const double *dij;     /* [nproj] projector strengths D_j (host) */
  int nocc;              /* occupied orbitals (closed shell, 2 electrons each) */
  const double *psi;     /* [nocc][npw_h] complex occupied orbitals, orthonormal and real in r,
                            (host or device); NULL: the library computes them (wdf_ground_state) */
  const double *eps;     /* [nocc] their eigenvalues (host); NULL when psi is NULL */
  int mem;               /* wdf_mem of vloc_r, beta and psi */
} wdf_system;

typedef struct wdf_options {
  int precision;     /* wdf_precision, default WDF_MIXED */
  int precond;       /* wdf_precond, default WDF_PRECOND_TPA */
  double cg_tol;     /* stop a solve at ||b - A x|| <= cg_tol ||b|| (default 1e-8) */
  int cg_maxiter;    /* CG iterations per solve, summed over refinement steps (default 1000) */
  double inner_tol;  /* WDF_MIXED: relative reduction asked of each FP32 inner solve (1e-5) */
  double alpha;      /* shift of the occupied space in the Sternheimer operator; <= 0: auto
                        (eps_max - eps_min + 1 hartree) */
  int max_batch;     /* most Sternheimer solves resident at once (0: all of a block) */
  double gs_tol;     /* ground state: residual norm per orbital (default 1e-10) */
  int gs_maxiter;    /* ground state Davidson iterations (default 300) */
  int gs_extra;      /* ground state: extra states beyond nocc carried in the Davidson (default 8) */
  void *stream;      /* cudaStream_t for all work of the context (NULL: default stream) */
  int device;        /* CUDA device ordinal (default 0) */
  int warm_start;    /* WDF_PRECOND_LEARNED: start each solve from the model's first iterate
                        x0 = o1(v, G) K b instead of 0 (default 0) */
  int residual_update; /* WDF_MIXED, WDF_MIXED_DF: after a batch's first full residual, take the
                        residual of x + d as r - A d with A d in FP32 and its error bound
                        eps_A ||d|| added to the stopping test, while that bound stays below
                        cg_tol ||b|| / 10 (eps_A: 16 x the batch's largest measured
                        ||A x - A_32 x|| / ||x||); 0 (default): every refinement recomputes
                        b - A x in the residual precision */
} wdf_options;

/* Statistics of the last apply / Davidson call. */
typedef struct wdf_stats {
  int64_t nsolve;          /* Sternheimer solves done */
  int64_t cg_iters;        /* CG iterations summed over solves (inner FP32 + FP64) */
  int32_t cg_iters_max;    /* most iterations of one solve */
  int32_t refinements;     /* WDF_MIXED: FP64 residual evaluations per solve, maximum */
  double max_residual;     /* largest final ||b - A x|| / ||b|| over solves (FP64) */
  int64_t napply;          /* chi0bar applications (perturbation vectors) */
  int32_t davidson_iters;  /* Davidson iterations */
  int32_t converged;       /* 1 if every requested quantity met its tolerance */
  double ms;               /* wall time of the call, milliseconds */
  int32_t fallbacks;       /* WDF_PRECOND_LEARNED: solves that stalled and restarted with TPA */
} wdf_stats;

/* Fill *opt with the defaults listed above. */
void wdf_default_options(wdf_options *opt);

/* Create a context: validate and copy the system to the GPU, build the plane-wave layout and
 * FFT plans, and, if sys->psi is NULL, compute the nocc lowest eigenpairs of H (Eq. (1)) by the
 * library's block Davidson with the TPA preconditioner to opt->gs_tol.
 * out: receives the context (NULL on failure). opt: NULL for defaults.
 * Errors: WDF_EINVAL (sizes, Miller set not a half sphere, grid too small for the sphere or not
 * 2,3,5-smooth), WDF_ENOMEM, WDF_ECUDA, WDF_ESTATE (no usable GPU), WDF_ENOCONV (ground state
 * did not converge: the context is still created and usable), WDF_ENAN. */
int wdf_setup_hamiltonian(wdf_ctx **out, const wdf_system *sys, const wdf_options *opt);

/* The canonical Gamma half sphere of {G : |G|^2 <= ecut} (ecut in bohr^-2) for the cell with
 * lattice vectors as rows: Miller triples with n3 > 0, or n3 = 0 and n2 > 0, or n3 = n2 = 0 and
 * n1 >= 0, ordered by |G|^2 (shells equal to 1e-9 ecut count as one) and then by (n1, n2, n3);
 * G = 0 first. This is the order wdf_system.miller expects. Host only (no GPU needed).
 * miller: NULL to query the count, else room for *npw_h triples. *npw_h: in, the room; out,
 * the count. Errors: WDF_EINVAL (singular cell, ecut <= 0, too little room). */
int wdf_half_sphere(const double cell[9], double ecut, int32_t *miller, int *npw_h);

/* Copy the context's Miller triples [npw_h][3] (host). */
int wdf_get_gvectors(const wdf_ctx *ctx, int32_t *miller);

/* Make a failed context usable again when the failure did not leave the device faulted (a
 * refused launch, an expired bounded wait): clears the error and returns WDF_OK; WDF_ESTATE
 * when the device reports a fault (then only wdf_destroy remains). */
int wdf_reset_error(wdf_ctx *ctx);

/* Release the context and all its device memory. NULL is ignored. */
void wdf_destroy(wdf_ctx *ctx);

/* Copy the occupied eigenpairs into eps[nocc] (host) and, if psi is not NULL, psi[nocc][npw_h]
 * complex (host or device per mem). Orbitals are real in r and orthonormal. */
int wdf_get_orbitals(wdf_ctx *ctx, double *eps, double *psi, int mem);

/* Apply H (Eq. (1): kinetic + local + Kleinman-Bylander) to nvec half-sphere vectors.
 * in, out: [nvec][npw_h] complex, host or device per mem; out may alias in. */
int wdf_apply_hamiltonian(wdf_ctx *ctx, int nvec, const double *in, double *out, int mem);

/* Switch wdf_options.residual_update of a live context (0 or 1). Errors: WDF_EINVAL. */
int wdf_set_residual_update(wdf_ctx *ctx, int on);

/* Apply the operator of the Sternheimer equations of Sec. 2.1, A_v = H - eps_v + alpha P (P the
 * projector on the occupied space, alpha the shift of wdf_options), to nvec half-sphere vectors,
 * vector k with v = vidx[k], in the precision the library computes residuals b - A x in: FP64
 * for WDF_FP64 and WDF_MIXED; double-float (about 48 significant bits, the projections on
 * [beta; psi] on the tensor cores by exact integer digits) for WDF_MIXED_DF.
 * vidx: [nvec] (host), each in [0, nocc). in, out: [nvec][npw_h] complex, host or device per
 * mem; out may alias in. Errors: WDF_EINVAL (bad sizes, NULL buffers, vidx out of range),
 * WDF_ETIMEOUT (a tensor-core kernel gave up waiting; out is then undefined). */
int wdf_apply_sternheimer_operator(wdf_ctx *ctx, int nvec, const int32_t *vidx, const double *in, double *out, int mem);

/* Solve the Sternheimer equations of Sec. 2.1 for nsolve right-hand sides:
 * (H - eps_v + alpha P) x_k = rhs_k with v = vidx[k], P the projector on the occupied space,
 * to ||rhs_k - A x_k|| <= cg_tol ||rhs_k||. For rhs_k orthogonal to the occupied space this is
 * the unique solution of (H - eps_v) x = rhs in that complement.
 * vidx: [nsolve] (host), each in [0, nocc). rhs, x: [nsolve][npw_h] complex (host or device).
 * st: optional statistics. Errors: WDF_EINVAL, WDF_ENOCONV (x holds the last iterate). */
int wdf_sternheimer(wdf_ctx *ctx, int nsolve, const int32_t *vidx, const double *rhs, double *x,
                    int mem, wdf_stats *st);

/* chi0bar phi for npert perturbations (Sec. 2.1: chi0bar = v^1/2 chi0 v^1/2 with the density
 * response by DFPT). For each perturbation p and occupied orbital v: dV_p = v^1/2 phi_p in real
 * space, one Sternheimer solve (H - eps_v) dpsi_vp = -Q dV_p psi_v to cg_tol, then
 * drho_p = 4 sum_v psi_v dpsi_vp and out_p = v^1/2 drho_p, v^1/2(G) = sqrt(4 pi)/|G|, zero at
 * G = 0.
 * phi: [npert][npw_h] complex, orthonormal or not; the G = 0 entry is ignored.
 * out: [npert][npw_h] complex = chi0bar phi; may alias phi. drho: optional [npert][npw_h]
 * complex plane-wave coefficients <b_G|drho_p>. All host or device per mem.
 * Errors: WDF_EINVAL, WDF_ENOMEM, WDF_ECUDA, WDF_ENOCONV (outputs from the last iterates). */
int wdf_apply_chi0(wdf_ctx *ctx, int npert, const double *phi, double *out, double *drho, int mem,
                   wdf_stats *st);

/* W_p x for nvec vectors from PDEP eigenpairs: the low-rank form of Eq. (5) without the
 * long-range term Xi, W_p = v^1/2 chibar v^1/2 with chibar = sum_a phibar_a lambda_a / (1 - lambda_a)
 * phibar_a^dagger (phibar orthonormal coefficient vectors, as wdf_pdep_davidson returns them; the
 * 1/Omega of Eq. (5) belongs to the paper's real-space normalisation of the eigenpotentials).
 * lambda: [neig] host, each < 1. phibar: [neig][npw_h]; in, out: [nvec][npw_h] complex, host or
 * device per mem; out may alias in. Errors: WDF_EINVAL. */
int wdf_apply_wp(wdf_ctx *ctx, int neig, const double *lambda, const double *phibar, int nvec, const double *in,
                 double *out, int mem);

/* chi0bar for several systems at once (batching form): out[k] = chi0bar phi[k] for context
 * ctx[k] and npert[k] perturbations, exactly as wdf_apply_chi0 would compute it. The systems run
 * concurrently, one host thread per system, each on its context's stream (a context on the
 * legacy default stream gets a private stream for the call), so that systems too small to fill
 * the GPU overlap. Contexts must be distinct and on one GPU; phi[k], out[k] host or device per
 * mem. st: NULL or an array of nsys statistics. Returns WDF_OK, the first error of a system, or
 * WDF_ENOCONV when every system finished but one did not converge; wdf_last_error(NULL) names
 * the failing system. */
int wdf_apply_chi0_multi(int nsys, wdf_ctx *const *ctx, const int *npert, const double *const *phi,
                         double *const *out, int mem, wdf_stats *st);

/* PDEP: the neig algebraically lowest eigenpairs of chi0bar (Eq. (5): lambda_a, phibar_a) by
 * block Davidson. Start block: the nguess vectors of guess (G = 0 entries ignored), at least
 * neig of them; expansion by the residuals of the unconverged Ritz pairs, two-pass classical
 * Gram-Schmidt in FP64 (vectors below 1e-12 after projection dropped), restart from the neig
 * Ritz vectors when the basis would exceed nbasis_max (0: 4*neig); converged when
 * ||chi0bar x_a - lambda_a x_a|| <= tol for all a.
 * lambda: [neig] ascending (host). phibar: [neig][npw_h] complex orthonormal (host or device).
 * Errors: WDF_EINVAL, WDF_ENOCONV (best Ritz pairs returned), others as wdf_apply_chi0. */
int wdf_pdep_davidson(wdf_ctx *ctx, int neig, int nbasis_max, int maxiter, double tol,
                      int nguess, const double *guess, double *lambda, double *phibar, int mem,
                      wdf_stats *st);

/* wdf_pdep_davidson from neig start vectors drawn by the library: Gaussian real and imaginary
 * parts from splitmix64(seed) (Steele, Lea, Flood 2014) with Box-Muller, G = 0 removed, each
 * scaled to unit norm. lambda host; phibar host or device per mem. */
int wdf_pdep_davidson_seeded(wdf_ctx *ctx, int neig, int nbasis_max, int maxiter, double tol, uint64_t seed,
                             double *lambda, double *phibar, int mem, wdf_stats *st);

/* A caller's operator for wdf_davidson: out = A in for nvec half-sphere vectors, in and out
 * [nvec][npw_h] complex in DEVICE memory of the context's GPU, owned by the library and valid
 * for the duration of the call (out arrives zeroed). The callback runs on the thread that called
 * wdf_davidson, after the library's stream has finished writing in; its results must be in out
 * when it returns (synchronise whatever stream it used). Return 0, or non-zero to abort the
 * eigensolve (wdf_davidson then returns WDF_EINVAL). */
typedef int (*wdf_operator_fn)(void *user, int nvec, const double *in, double *out);

/* The library's block Davidson on a caller's operator (Sec. 3.3: one Davidson solver serves PDEP
 * and the BSE and TDDFT eigenproblems): the neig algebraically lowest eigenpairs of A, a
 * Hermitian operator on the context's plane-wave basis that maps real functions to real
 * functions (symmetric in the Gamma inner product). Same algorithm, restart rule and convergence
 * test as wdf_pdep_davidson (||A x_a - lambda_a x_a|| <= tol), with apply(user, ...) in place of
 * chi0bar. zero_g0: 1 keeps the G = 0 component out of the space (as for chi0bar), 0 keeps it.
 * guess: [nguess][npw_h] start block (nguess >= neig), host or device per mem; lambda: [neig]
 * ascending (host); vec: [neig][npw_h] orthonormal eigenvectors, host or device per mem.
 * st: napply, davidson_iters, converged and ms are filled. Errors: WDF_EINVAL (arguments, or the
 * callback failed), WDF_ENOCONV (best Ritz pairs returned), others as wdf_pdep_davidson. */
int wdf_davidson(wdf_ctx *ctx, wdf_operator_fn apply, void *user, int neig, int nbasis_max, int maxiter, double tol,
                 int zero_g0, int nguess, const double *guess, double *lambda, double *vec, int mem, wdf_stats *st);

/* Bytes of the device array behind wdf_apply_hamiltonian_noalloc: 64 MiB, present on every GPU
 * that loads the library for the life of the process. */
#define WDF_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* H x for nvec vectors, the same result as wdf_apply_hamiltonian, without allocating any device
 * memory. For callers that cannot call cudaMalloc: processes whose device memory is owned by
 * another allocator (a framework's caching pool, whose accounting an outside allocation would
 * break), or services with a fixed device memory budget. The paper has no counterpart: this
 * entry point only changes where the temporaries live. All of them come from one file-scope
 * device array of WDF_NOALLOC_SCRATCH_BYTES; a call that would need more (about 0.7 MB per vector
 * for a 64^3 grid with 8,440 plane waves) returns WDF_EINVAL and asks for fewer vectors per call.
 * in, out: [nvec][npw_h] complex in DEVICE memory of the context's GPU (checked: anything else
 * is WDF_EINVAL); out may equal in (the input is read in full before any output is written).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it, so make that first call before any stream capture. Every call on a device shares
 * the array: calls whose GPU work may overlap (different streams without ordering) race.
 * Returns after the result is in out. Errors: WDF_EINVAL, WDF_ECUDA, WDF_ESTATE. */
int wdf_apply_hamiltonian_noalloc(wdf_ctx *ctx, int nvec, const double *in, double *out);

/* ---------------------------------------------------------------------------------------------
 * Learned Sternheimer preconditioner. The paper has no counterpart: it is an extension that
 * keeps the method's result (the converged solves) and changes only the CG path to it.
 *
 * Model: a multilayer perceptron 4 -> 64 -> 64 -> 2 (tanh hidden layers) evaluated per occupied
 * orbital v and plane wave G on the features
 *   f0 = log(1 + (1/2 |G|^2) / T_v), f1 = eps_v, f2 = T_v, f3 = log(npw_h |c_v(G)|^2 + 1e-6),
 * normalised as (f - mu) / sd; T_v is the kinetic energy of psi_v. Output o0 gives the diagonal
 * scale s = exp(o0) (o0 clamped to [-8, 8]) of the preconditioner s K_TPA; output o1 the first
 * iterate x0 = o1 K_TPA b.
 * Training samples come from converged TPA solves of chi0bar applications: per (v, G), summed
 * over the solves of orbital v, E_x = sum |x|^2, E_k = sum |K b|^2, C = sum Re(conj(K b) x);
 * targets t0 = 1/2 log(E_x / E_k), t1 = C / E_k; weights w0 ~ E_x + E_k, w1 ~ E_k counted for G
 * and -G and normalised to unit sum per call. Loss sum_i sum_k w_ik (o_ik - t_ik)^2; full-batch
 * Adam (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) by the library's own kernels.
 * Weights: WDF_MODEL_FLOATS floats W1[4][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2]
 * (the WDF_MODEL_NPARAM trained values), then mu[4], sd[4].
 * Samples: features [n][4], targets [n][2], weights [n][2], floats.
 * A model lives on one GPU and is used by one thread at a time. */
typedef struct wdf_model wdf_model;
#define WDF_MODEL_NPARAM 4610
#define WDF_MODEL_FLOATS 4618

typedef struct wdf_train_opts {
  int steps;       /* full-batch Adam steps per wdf_model_train call (default 600) */
  double lr;       /* Adam learning rate (default 3e-3) */
  int npert;       /* wdf_train_preconditioner: perturbations per context (default 8) */
  uint64_t seed;   /* wdf_train_preconditioner: seed of the perturbations and initial weights */
} wdf_train_opts;

typedef struct wdf_train_stats {
  int64_t nsamples;   /* samples in the model */
  int32_t steps;      /* Adam steps taken by the call */
  double loss_first;  /* loss before the first step of the call */
  double loss_last;   /* loss before the last step of the call */
  double ms;          /* wall time of the call, milliseconds */
} wdf_train_stats;

void wdf_default_train_opts(wdf_train_opts *opt);

/* New model on CUDA device `device`: weights drawn from splitmix64(seed) (normal, variance
 * 1/fan-in; biases 0), mu = 0, sd = 1, no samples. The first wdf_model_train call of a model
 * created this way sets mu, sd from the samples and b3 to the weighted target means.
 * Errors: WDF_EINVAL, WDF_ENOMEM, WDF_ECUDA, WDF_ESTATE. */
int wdf_model_create(int device, uint64_t seed, wdf_model **out);
/* Release a model (NULL is ignored). */
void wdf_model_free(wdf_model *m);
/* Replace / read the WDF_MODEL_FLOATS weights (host). Setting weights keeps mu and sd as given
 * and resets the Adam moments. */
int wdf_model_set_weights(wdf_model *m, const float *w);
int wdf_model_get_weights(const wdf_model *m, float *w);
/* Apply chi0bar to npert perturbations phi ([npert][npw_h] complex, host or device per mem) with
 * TPA solves to the context's cg_tol and append the nocc * npw_h samples of those solves, in the
 * order (v, half-sphere index). The model must live on the context's GPU. st: optional stats of
 * the chi0bar application. Errors: as wdf_apply_chi0. */
int wdf_model_add_solves(wdf_model *m, wdf_ctx *ctx, int npert, const double *phi, int mem, wdf_stats *st);
/* Number of samples (-1 for NULL). */
int64_t wdf_model_num_samples(const wdf_model *m);
/* Replace all samples by n given ones / read count samples from index first (host arrays). */
int wdf_model_set_samples(wdf_model *m, int64_t n, const float *feat, const float *tgt, const float *wt);
int wdf_model_get_samples(const wdf_model *m, int64_t first, int64_t count, float *feat, float *tgt, float *wt);
/* Loss over all samples and its gradient grad[WDF_MODEL_NPARAM] (host) at the current weights. */
int wdf_model_loss_grad(wdf_model *m, double *loss, double *grad);
/* opt->steps full-batch Adam steps on the samples (opt NULL: defaults). Errors: WDF_EINVAL (no
 * samples), WDF_ENAN (non-finite loss). */
int wdf_model_train(wdf_model *m, const wdf_train_opts *opt, wdf_train_stats *st);
/* Outputs out[n][2] = (o0, o1) for raw features feat[n][4] (host). */
int wdf_model_predict(wdf_model *m, int64_t n, const float *feat, float *out);
/* Evaluate the model for every (v, G) of the context, store s K_TPA and o1 K_TPA, and switch the
 * context to WDF_PRECOND_LEARNED. m NULL: back to WDF_PRECOND_TPA. The model must live on the
 * context's GPU; the context keeps no reference to it. */
int wdf_set_model(wdf_ctx *ctx, const wdf_model *m);
/* Convenience: create a model from opt->seed, add the solves of opt->npert perturbations drawn
 * from splitmix64(opt->seed) (Gaussian coefficients, G = 0 removed, unit norm) for each of the n
 * contexts, and train it. *out receives the model (NULL on failure). */
int wdf_train_preconditioner(wdf_ctx *const *ctx, int n, const wdf_train_opts *opt, wdf_model **out,
                             wdf_train_stats *st);

/* Instrumentation: time one kernel class with CUDA events. Every later launch of that class made
 * by calls on ctx is bracketed by two events recorded on the stream it is launched on.
 * kernel: a class name, optionally with ":64", ":32" or ":48" for the precision, e.g. "plane_vloc:32".
 * Precision suffixes: 64 (FP64), 32 (FP32), 48 (double-float). Classes: zpass_g2r, zpass_r2g, plane_vloc, plane_g2r, plane_prod, plane_accum, gram, gram_sum,
 * lincomb, dot_partial, cg_start, cg_update, cg_direction, cg_scalars, axpby, scale_rows,
 * convert, ext_to_int, int_to_ext, ritz_residual, tpa_table, kinetic, mul_table, check_finite,
 * jac_init, jac_rows, jac_cols, jac_check, jac_sort, split_pairs, scale_elems, gather_shift,
 * sum_chunks, chol_inv, compact, tc_prep, mlp_predict, mlp_grad, mlp_reduce, mlp_adam, mlp_table, mlp_accum, mlp_samples. NULL stops timing. Calling it resets the counters. Errors: WDF_EINVAL. */
int wdf_profile_kernel(wdf_ctx *ctx, const char *kernel);

/* Launches of the selected class since wdf_profile_kernel and their summed device time in
 * milliseconds. Synchronises the context's stream. */
int wdf_profile_read(wdf_ctx *ctx, int64_t *launches, double *ms);

/* Work units of the timed launches of the selected class since wdf_profile_kernel: thread blocks
 * for kernels that give each block one unit, and for plane_vloc the (pair of solves, z plane)
 * units whichever kernel runs it (the persistent variant loops over several units per block).
 * Does not synchronise. */
int wdf_profile_units(wdf_ctx *ctx, int64_t *blocks);

/* The V_loc plane kernel chosen at setup by timing for the given arithmetic (bits = 32 FP32,
 * 64 FP64, 48 double-float): 1 register lines, 2 Stockham, 3 generic, 4 two-thread register
 * lines, 5 persistent with bulk copies; 0 when that arithmetic has no V_loc plane kernel in this
 * context (WDF_EINVAL for other bits). Instrumentation: lets a caller match kernel counters taken
 * on one variant to the kernel that runs. */
int wdf_plane_variant(const wdf_ctx *ctx, int bits, int *variant);

/* Number of kernel launches the library has made in this process so far (all contexts). */
int64_t wdf_launch_count(void);

/* Device memory held by the library (no counterpart in the paper: accounting for services that
 * run under a memory budget). Workspaces are grow-only buffers per context and model.
 * wdf_device_bytes: bytes those buffers hold now, over all contexts and models of the process
 *   (the static array behind wdf_apply_hamiltonian_noalloc is not counted).
 * wdf_alloc_count: cudaMalloc calls the library has made for them so far.
 * wdf_set_device_limit: cap on the bytes held; a call that would grow a buffer past it returns
 *   WDF_ENOMEM without allocating, and its context stays usable (a later call with a higher
 *   cap, or with a smaller block, succeeds). bytes <= 0: no cap (the default). Process-wide. */
int64_t wdf_device_bytes(void);
int64_t wdf_alloc_count(void);
void wdf_set_device_limit(int64_t bytes);

/* Polls a software device wait makes before it gives up: the grid barrier of the cooperative
 * form of the subspace eigensolver (used when the cluster form is unavailable or disabled with
 * the environment variable WDF_NO_CLUSTER_JACOBI). On expiry the waiting blocks set the
 * context's error flag and return, and the call returns WDF_ETIMEOUT with the context still
 * usable. polls <= 0 restores the default (2^24). For tests of the timeout path and for
 * callers that prefer an early error to a long stall. Errors: WDF_EINVAL (NULL context). */
int wdf_set_wait_limit(wdf_ctx *ctx, int64_t polls);

/* Static text for a status code. */
const char *wdf_strerror(int status);

/* Message of the last failure in ctx (or of the last failed setup when ctx is NULL). */
const char *wdf_last_error(const wdf_ctx *ctx);

/* Library version string. */
const char *wdf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WDF_H */

// Kernel launchers of libwdf.so (internal interface between the engine and the kernels).
#pragma once

#include "common.cuh"

namespace wdf {

constexpr int kZCols = 16;  // rep columns per block of the n3 transforms

enum { EPI_STORE = 0, EPI_HSHIFT = 1, EPI_DRHO = 2 };
enum { OP_VLOC = 0, OP_G2R = 1, OP_PROD_R2G = 2, OP_ACCUM = 3 };

// Everything an FFT launch needs for one precision.
template <typename T> struct FftCtx {
  Geo g;
  Plan1D P1, P2, P3;
  const cplx<T> *tw1, *tw2, *tw3;  // exp(2 pi i t / n) per axis
  const int *jidx;                 // [n2][n1] disk column at natural (y, x), or -1
  const int *jnat;                 // [ndisk] natural y * n1 + x of each disk column
  int vloc_variant = 0;            // V_loc plane kernel: 0 default order, 1 register, 2 Stockham, 3 generic,
                                   // 4 register with two threads per line (n1 = n2 = 64), 5 persistent
                                   // with bulk copies (64 x 64 planes with a full disk), 6 double-float
                                   // one task per thread (64 x 64), 7 persistent with two threads per
                                   // line (96 x 96 planes with a full disk)
  int *err = nullptr;              // device flag set by a kernel whose bounded wait expired
};

template <typename T> struct EpiArgs {
  cplx<T> *Y = nullptr;         // output vectors (EPI_STORE / EPI_HSHIFT), drho (EPI_DRHO)
  cplx<T> *Y2 = nullptr;        // EPI_DRHO: v^1/2 drho
  const cplx<T> *X = nullptr;   // EPI_HSHIFT: the transformed vectors themselves
  const double *shift = nullptr;  // EPI_HSHIFT: per-vector shift (eps_v)
  const double *vhalf = nullptr;  // EPI_DRHO: v^1/2 per element
  T scale = 1;                  // applied to the unpacked values
};

template <typename T> struct PlaneArgs {
  cplx<T> *cb = nullptr;        // column buffer (in and out)
  cplx<T> *cb2 = nullptr;       // OP_ACCUM output column buffer (per perturbation pair)
  const T *field = nullptr;     // OP_VLOC: V_loc grid; OP_PROD_R2G / OP_ACCUM: psi_v(r) grids
  cplx<T> *grid = nullptr;      // OP_G2R out; OP_PROD_R2G in (dV pairs); OP_ACCUM accumulator
  int nocc = 0;
};

template <typename T> void set_fft_smem_limits(const Geo &g);
// plane kernels specialised for compile-time sizes (plane_fast.cu); false when not available
bool plane_fast_supported(int n1, int n2);
template <typename T> void set_plane_fast_limits(const Geo &g);
template <typename T> bool launch_plane_fast(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st);
// whether V_loc plane variant v (1 register, 2 Stockham, 3 generic, 4 two-thread register,
// 5 persistent with bulk copies, 6 double-float one task per thread) exists
template <typename T> bool plane_variant_available(const FftCtx<T> &f, int v);
constexpr int kPlaneVariants = 7;  // variants are numbered 1 .. kPlaneVariants
// whether the orbital sum of the density response runs as G2R transforms + k_orbital_sum
template <typename T> bool plane_accum_by_g2r(const FftCtx<T> &f);
// acc[i] = sum_v psir[v][i] fields[v][i] over the ngrid points, orbitals in order
template <typename R>
void launch_orbital_sum(const cplx<R> *fields, const R *psir, int nocc, size_t ngrid, cplx<R> *acc, cudaStream_t st);
// x[i] = value
template <typename R> void launch_fill(R *x, size_t count, double value, cudaStream_t st);
// persistent FP32 V_loc plane kernel (plane_pipe.cu); false when the geometry has no instance
bool plane_pipe_available(const Geo &g, const int *err);
void set_plane_pipe_limits(const Geo &g);
bool launch_plane_pipe(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st);
// persistent FP32 V_loc plane kernel with two threads per line (plane_pipe2.cu; 96 x 96 planes)
bool plane_pipe2_available(const Geo &g, const int *err);
void set_plane_pipe2_limits(const Geo &g);
bool launch_plane_pipe2(const FftCtx<float> &f, int npair, const PlaneArgs<float> &pa, cudaStream_t st);
// compile-time Stockham plane kernels for the further sizes (plane_more_*.cu): float, and
// double-float in two size groups; false when the size is not in the group
bool launch_plane_more_f32(const FftCtx<float> &f, int op, int nblk, const PlaneArgs<float> &pa, cudaStream_t st);
void set_plane_more_limits_f32(const Geo &g);
bool launch_plane_more_df_a(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st);
void set_plane_more_limits_df_a(const Geo &g);
bool launch_plane_more_df_b(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st);
void set_plane_more_limits_df_b(const Geo &g);
// double-float 64 x 64 plane kernel (plane_df.cu) for OP_VLOC, OP_PROD_R2G and OP_ACCUM
bool plane_df_available(const Geo &g, const int *jidx);
void set_plane_df_limits(const Geo &g);
bool launch_plane_df(const FftCtx<df64> &f, int op, int nblk, const PlaneArgs<df64> &pa, cudaStream_t st);
template <typename T> size_t plane_smem(const Geo &g);
template <typename T> size_t zpass_smem(const Geo &g);
// CG direction update folded into the first transform: p = K r + beta p for active solves
template <typename T> struct PDir {
  cplx<T> *p = nullptr;          // also the transformed vectors
  const cplx<T> *r = nullptr;
  const T *K = nullptr;          // [nocc][ld] preconditioner, or null (identity)
  const int *vidx = nullptr, *active = nullptr;
  const double *beta = nullptr;
};
template <typename T> void launch_zpass_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T>
void launch_zpass_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T>
void launch_zpass_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st);
template <typename T> void launch_plane(const FftCtx<T> &f, int op, int nblk, const PlaneArgs<T> &pa, cudaStream_t st);
// compile-time n3 transforms (zpass_fast_*.cu); false when the size has none
template <typename T> bool zpass_fast_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T> bool zpass_fast_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T>
bool zpass_fast_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st);
template <typename T> void set_zpass_fast_limits(const Geo &g);
// the further sizes (zpass_more_*.cu: float and double-float)
template <typename T> bool zpass_more_g2r(const FftCtx<T> &f, const cplx<T> *X, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T> bool zpass_more_g2r_dir(const FftCtx<T> &f, const PDir<T> &d, int nvec, cplx<T> *cb, cudaStream_t st);
template <typename T>
bool zpass_more_r2g(const FftCtx<T> &f, int epi, const cplx<T> *cb, int nvec, const EpiArgs<T> &ea, cudaStream_t st);
template <typename T> void set_zpass_more_limits(const Geo &g);

// ---------------------------------------------------------------------------------------------
// dense linear algebra on blocks of internal vectors (rows of length ld, nint live elements)

// out[i * ldo + j] = <A_i, B_j> = sum_e w_e Re(conj(A_i[e]) B_j[e]), w = 1 on column (0,0), else 2.
// work: scratch for split partial sums, gram_work_doubles() long (without it no split is used).
template <typename T>
void launch_gram(const Geo &g, const cplx<T> *A, int na, const cplx<T> *B, int nb, double *out, int ldo, double *work,
                 size_t work_cap, cudaStream_t st);
size_t gram_work_doubles(const Geo &g, int na, int nb, int ldo);
// Y_s = c0 Y_s + sum_j U_j C[j * ldc + s] d_j   (d may be null: d_j = 1), s < ny, j < nu.
template <typename T>
void launch_lincomb(const Geo &g, cplx<T> *Y, int ny, const cplx<T> *U, int nu, const double *C, int ldc,
                    const double *d, double c0, cudaStream_t st);
// launch_lincomb plus partial inner products <P_s, Y_s> of the results, written to
// part[s * lincomb_dot_chunks(g) + block]; returns false (nothing launched) for ny <= 8
template <typename T>
bool launch_lincomb_dot(const Geo &g, cplx<T> *Y, int ny, const cplx<T> *U, int nu, const double *C, int ldc, const double *d,
                        double c0, const cplx<T> *P, double *part, cudaStream_t st);
int lincomb_dot_chunks(const Geo &g);
// per-vector partial inner products: part[s * nchunk + c] over element chunk c
template <typename T>
void launch_dot_partial(const Geo &g, const cplx<T> *A, const cplx<T> *B, int nvec, double *part, int nchunk,
                        cudaStream_t st);
int dot_chunks(const Geo &g);
// part[s * nchunk + c] = sum over chunk c of w_e |A_s[e] - B_s[e]|^2 (A FP64, B FP32)
void launch_diff_partial(const Geo &g, const cplx<double> *A, const cplx<float> *B, int nvec, double *part, int nchunk, cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// CG state per solve (device arrays of length n unless noted)
struct CgState {
  double *rz, *rz_new, *pap, *rr;       // <r,z>, beta (after the scalar step), <p,Ap>, <r,r>
  double *thr;                           // stop a solve once <r,r> <= thr
  double *shift;                         // eps_v of each solve
  double *part1, *part2;                 // partial sums [n * nchunk]
  int *active;                           // 1 while the solve iterates
  int *iters;                            // iterations done
  int *nactive;                          // [1] count of active solves
  int *vidx;                             // preconditioner row of each solve (its orbital for TPA)
  // learned preconditioner only (krow null otherwise): rows [0, nocc) of the table are learned,
  // rows [nocc, 2 nocc) TPA; a solve whose <r,r> falls by less than 19% over 5 iterations (||r||
  // by less than 10%) moves to its TPA row and restarts with beta = 0
  int *krow = nullptr;                   // = vidx (the same array) when the table is learned
  const int *vorig = nullptr;            // orbital of each solve
  int nocc = 0;
  double *rr_ref = nullptr;              // <r,r> at the last stall check
  int *it_ref = nullptr;                 // iteration of the last stall check
  double *part3 = nullptr;               // partials of <r, K_TPA r> [n * nchunk]
  int *nfb = nullptr;                    // [1] solves moved to TPA
  // after compaction of the active solves: row i of the work arrays is solve home[i] of the
  // caller's x (null: identity)
  const int *home = nullptr;
};

// z = K r (TPA per orbital), p = z, and partials for <r,z>, <r,r>
template <typename T>
void launch_cg_start(const Geo &g, const cplx<T> *r, cplx<T> *z, cplx<T> *p, const T *kprec, const CgState &s, int n,
                     int nchunk, cudaStream_t st);
// alpha = rz / pAp; x += alpha p; r -= alpha Ap; z = K r; partials <r,z>, <r,r> (and, for the
// learned table, <r, K_TPA r> of the solves still on a learned row)
template <typename T>
void launch_cg_update(const Geo &g, cplx<T> *x, cplx<T> *r, cplx<T> *z, const cplx<T> *p, const cplx<T> *Ap,
                      const T *kprec, const CgState &s, int n, int nchunk, cudaStream_t st);
// p = z + beta p for active solves
template <typename T>
void launch_cg_direction(const Geo &g, cplx<T> *p, const cplx<T> *z, const CgState &s, int n, cudaStream_t st);
// reduce partials: which = 0 -> pap from part1; which = 1 -> new <r,z> from part1, rr from part2,
// then the stopping test rr <= thr, beta and iteration counting; which = 2: rz, rr at start
void launch_cg_scalars(const CgState &s, int n, int nchunk, int which, int maxiter, cudaStream_t st);

// elementwise helpers
template <typename T> void launch_axpby(const Geo &g, cplx<T> *y, const cplx<T> *x, int n, double a, double b, cudaStream_t st);
template <typename T> void launch_scale_rows(const Geo &g, cplx<T> *y, const double *coef, int n, cudaStream_t st);
template <typename Tin, typename Tout>
void launch_convert(const Geo &g, Tout *y, const Tin *x, size_t count, cudaStream_t st);
// external half-sphere vectors <-> internal layout
void launch_ext_to_int(const double *ext, int n, int npw_h, const int *emap, const int *emap2, const int *econj,
                       const double *scale_int, cplx<double> *out, int ld, cudaStream_t st);
void launch_int_to_ext(const cplx<double> *in, int n, int ld, int npw_h, const int *emap, const int *econj,
                       double *ext, cudaStream_t st);
// residual subtraction for Davidson: R_a = AX_a - theta_a X_a
void launch_ritz_residual(const Geo &g, cplx<double> *R, const cplx<double> *AX, const cplx<double> *X,
                          const double *theta, int n, cudaStream_t st);
// TPA preconditioner table K[v][e] = tpa(0.5 g2[e] / T_v)
template <typename T> void launch_mul_table(const Geo &g, cplx<T> *y, const T *tab, int n, cudaStream_t st);
template <typename T> void launch_tpa_table(const Geo &g, T *K, const double *tkin, int n, cudaStream_t st);
void launch_kinetic(const Geo &g, const cplx<double> *X, int n, double *tkin, cudaStream_t st);
// check for non-finite values; sets *flag = 1 if any
template <typename T> void launch_check_finite(const T *x, size_t count, int *flag, cudaStream_t st);

// Cholesky of an n x n SPD matrix and inverse of its factor in one block (n <= 160): writes the
// coefficients C = L^-T for launch_lincomb and *ok = 0 when a pivot is below tol * max diagonal
void launch_chol_inv(const double *G, int n, double *C, double tol, int *ok, cudaStream_t st);
size_t chol_inv_smem(int n);
void set_chol_inv_limits(int nmax);
constexpr int kCholMax = 160;  // n^2 + n doubles of shared memory (<= 227 KB)

// learned preconditioner (mlp.cu): weights W[kMlpFloats] = W1[4][64], b1, W2[64][64], b2, W3[64][2],
// b3 (kMlpParams trained values), mu[4], sd[4]; samples feat[n][4], tgt[n][2], wt[n][2]
constexpr int kMlpParams = 4610;
constexpr int kMlpFloats = 4618;
size_t mlp_grad_smem();
void set_mlp_limits();
int mlp_grad_blocks(long long n);
// out[0 .. kMlpParams) = gradient, out[kMlpParams] = loss; part: mlp_grad_blocks(n) * (kMlpParams + 1)
void launch_mlp_grad(const float *W, const float *feat, const float *tgt, const float *wt, long long n, double *part, double *out,
                     cudaStream_t st);
void launch_mlp_adam(double *w64, float *w32, const double *grad, double *m, double *v, int t, double lr, cudaStream_t st);
// m64/m32 [2 nocc][ld]: rows v = s(v,e) K(v,e), rows nocc + v = K(v,e); w64 [nocc][ld] = o1 K
void launch_mlp_table(const Geo &g, const float *W, const cplx<double> *psi, const double *tkin, const double *eps, int npw_h,
                      const double *ktpa, int nocc, double *m64, float *m32, double *w64, cudaStream_t st);
void launch_mlp_predict(const float *W, const float *feat, long long n, float *out, cudaStream_t st);
// sums [3][nocc][ld] += (|x|^2, |K b|^2, Re(conj(K b) x)) over the solves of a chi0bar block
void launch_mlp_accum(const Geo &g, const cplx<double> *b, const cplx<double> *x, int ns, int nocc, const double *ktpa, double *sums,
                      cudaStream_t st);
// nocc * npw_h samples (v-major, external order) from the sums; wraw: 2 n doubles, wsum: 2
void launch_mlp_samples(const Geo &g, const int *emap, int npw_h, int nocc, const double *sums, const cplx<double> *psi,
                        const double *tkin, const double *eps, float *feat, float *tgt, float *wt, double *wraw, double *wsum,
                        cudaStream_t st);

// tensor-core (tcgen05 kind::tf32, three-term split) projections of the FP32 CG (tc_gemm.cu);
// on unless WDF_NO_TC is set in the environment (then the CUDA-core kernels run)
bool tc_enabled();
int tc_rows(int na);  // rows of U rounded up to 32 (the MMA N of the projections, <= 256)
void set_tc_limits();
void launch_tc_prep_u(const Geo &g, const float2 *U, int na, float *uwh, float *uwl, float *uth, float *utl, cudaStream_t st);
// most rows of U ([beta; psi]) the tensor-core projections take (memory of the hi/lo copies only)
constexpr int kTcMaxRows = 4096;
size_t gram_tc_work_doubles(const Geo &g, int na, int nb);
// out[j][s] (ldo = nb) = sum_e w_e Re(conj(U_j) X_s) for j < na, s < nb
void launch_gram_tc(const Geo &g, const float *X, int nb, const float *uwh, const float *uwl, int na, double *out, double *work,
                    size_t work_cap, int *err, cudaStream_t st);
// Y_s = c0 Y_s + sum_j U_j S[j][s] d_j, partial <P_s, Y_s> per 128-element tile when part != null
void launch_lincomb_tc(const Geo &g, float *Y, int ny, const double *S, int ldc, const double *d, int na, float *chi, float *clo,
                       const float *uth, const float *utl, float c0, const float *P, double *part, int *err, cudaStream_t st);

// double-float projections on the tensor cores by exact integer digits (oz_gemm.cu); on with the
// tensor-core path unless WDF_NO_OZ is set in the environment
constexpr int OZ_DIGITS = 7;  // digits of 7 bits per value: a 49-bit fixed-point copy of each row
struct OzMat {
  uint16_t *dig = nullptr;  // [OZ_DIGITS][plane] bf16 digits: row r at dig + t plane + r kpad
  int *ex = nullptr;        // [rows] row exponents (every |value| < 2^ex)
  int rows = 0, kpad = 0;   // kpad: allocated values per row (a multiple of 32)
  size_t plane = 0;         // values between digit planes
  OzMat sub(int r0, int nr) const {
    OzMat m = *this;
    m.dig += (size_t)r0 * kpad;
    m.ex += r0;
    m.rows = nr;
    return m;
  }
};
bool oz_enabled();
int oz_kpad(int K);
void set_oz_limits();
// digits of rows of 2 N_int real values (complex rows of ld), times the Gamma-point weights when
// weighted
void launch_oz_rows_df(const Geo &g, const cplx<df64> *src, int rows, bool weighted, const OzMat &out, cudaStream_t st);
void launch_oz_rows_f64(const Geo &g, const cplx<double> *src, int rows, bool weighted, const OzMat &out, cudaStream_t st);
// digits of the transpose of src[j][c] (j < nj, c < ncol, row stride lds), row j scaled by d[j]
void launch_oz_cols(const double *src, size_t lds, int nj, int ncol, const double *d, const OzMat &out, cudaStream_t st);
size_t oz_gram_work_doubles(int na, int nb, int K);
// out[j][s] (row stride ldo) = sum_k U[j][k] X[s][k] over K values
void launch_oz_gram(const OzMat &U, const OzMat &X, int K, double *out, int ldo, double *work, size_t work_cap, int *err, cudaStream_t st);
// Y[s][f] = c0 Y[s][f] + sum_j C[s][j] Ut[f][j] over K values of j (double-float Y, row stride ldy
// double-floats; c0 in {-1, 0, 1})
void launch_oz_lincomb(const OzMat &C, const OzMat &Ut, int K, df64 *Y, size_t ldy, float c0, int *err, cudaStream_t st);

// symmetric eigensolver (cyclic Jacobi, parallel ordering) of an n x n matrix A (ld = n), FP64.
// On exit w holds eigenvalues ascending and V[i * n + k] the i-th component of eigenvector k.
// polls of the cooperative eigensolver's grid barrier before it gives up and flags the error
constexpr long kGridBarrierPolls = 1L << 24;
// wait_limit: polls of the cooperative form's grid barrier (<= 0: kGridBarrierPolls)
void jacobi_eigh(double *A, double *V, double *w, int n, double *work, int *iwork, cudaStream_t st, long wait_limit = 0);
size_t jacobi_work_doubles(int n);
void set_jacobi_limits(int nmax);  // shared memory of the cluster eigensolver for n <= nmax

}  // namespace wdf

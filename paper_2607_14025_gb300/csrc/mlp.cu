// Learned Sternheimer preconditioner: a multilayer perceptron 4 -> 64 -> 64 -> 2 evaluated per
// occupied orbital v and plane wave G, trained by full-batch Adam on samples taken from converged
// TPA solves. The paper has no such model; it changes the CG path only, never the solution.
//
// Kernels:
//   k_mlp_grad     loss and gradient over all samples, one 128-sample tile per step of a block:
//                  forward and backward per thread (hidden layer 1 in registers), then the weight
//                  gradients of the tile as sums over its samples from shared memory; per-block
//                  FP64 partial gradients
//   k_mlp_reduce   fixed-order sum of the block partials (deterministic)
//   k_mlp_adam     Adam update in FP64 of the master weights, FP32 copy for the kernels
//   k_mlp_table    the per-(v, G) preconditioner s K_TPA and first-iterate gain o1 K_TPA
//   k_mlp_accum    E_x, E_k, C per (v, G) from a batch of converged solves
//   k_mlp_samples  features, targets and raw weights per (v, half-sphere G) from those sums
#include <cmath>

#include "engine.cuh"

namespace wdf {

namespace {

constexpr int MH = 64;                       // hidden width
constexpr int OW1 = 0, OB1 = 256, OW2 = 320, OB2 = 4416, OW3 = 4480, OB3 = 4608;
constexpr int OMU = kMlpParams, OSD = kMlpParams + 4;
static_assert(OB3 + 2 == kMlpParams, "parameter layout");
static_assert(OSD + 4 == kMlpFloats, "model layout");

constexpr int TS = 128;  // samples per tile = threads per block of k_mlp_grad
constexpr int P65 = 65;  // padded row of the per-sample activations (conflict-free columns)
constexpr int P68 = 68;  // padded row that keeps float4 alignment

struct MlpW {
  float w1[4 * MH];   // [k][i]
  float b1[MH];
  float w2t[MH * MH];  // transposed: [j][i] = W2[i][j]
  float b2[MH];
  float w3[MH * 2];   // [j][k]
  float b3[2];
  float mu[4], sd[4];
};

struct TrainSmem {
  MlpW w;
  float H1[TS * P65], H2[TS * P65], D1[TS * P65];
  __align__(16) float D2[TS * P68];
  float X[TS * 4], E[TS * 2];
  double g[kMlpParams + 1];  // this block's gradient, then its loss
  double red[TS / 32];
};

__device__ void load_weights(MlpW &s, const float *__restrict__ W) {
  for (int t = threadIdx.x; t < 4 * MH; t += blockDim.x) s.w1[t] = W[OW1 + t];
  for (int t = threadIdx.x; t < MH; t += blockDim.x) {
    s.b1[t] = W[OB1 + t];
    s.b2[t] = W[OB2 + t];
  }
  for (int t = threadIdx.x; t < MH * MH; t += blockDim.x) {
    const int i = t / MH, j = t % MH;
    s.w2t[j * MH + i] = W[OW2 + t];
  }
  for (int t = threadIdx.x; t < 2 * MH; t += blockDim.x) s.w3[t] = W[OW3 + t];
  if (threadIdx.x < 2) s.b3[threadIdx.x] = W[OB3 + threadIdx.x];
  if (threadIdx.x < 4) {
    s.mu[threadIdx.x] = W[OMU + threadIdx.x];
    s.sd[threadIdx.x] = W[OSD + threadIdx.x];
  }
}

// hidden layer 1 of one sample into registers (x already normalised)
__device__ __forceinline__ void layer1(const MlpW &s, const float x[4], float h1[MH]) {
#pragma unroll
  for (int i = 0; i < MH; ++i) {
    float a = s.b1[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) a = fmaf(x[k], s.w1[k * MH + i], a);
    h1[i] = tanhf(a);
  }
}

// pre-activation of hidden unit j of layer 2: b2[j] + sum_i h1[i] W2[i][j] (two partial chains)
__device__ __forceinline__ float layer2_pre(const MlpW &s, const float h1[MH], int j) {
  const float4 *wr = reinterpret_cast<const float4 *>(s.w2t + j * MH);
  float a0 = s.b2[j], a1 = 0.f;
#pragma unroll
  for (int q = 0; q < MH / 4; q += 2) {
    const float4 u = wr[q], v = wr[q + 1];
    a0 = fmaf(h1[4 * q + 0], u.x, a0);
    a1 = fmaf(h1[4 * q + 4], v.x, a1);
    a0 = fmaf(h1[4 * q + 1], u.y, a0);
    a1 = fmaf(h1[4 * q + 5], v.y, a1);
    a0 = fmaf(h1[4 * q + 2], u.z, a0);
    a1 = fmaf(h1[4 * q + 6], v.z, a1);
    a0 = fmaf(h1[4 * q + 3], u.w, a0);
    a1 = fmaf(h1[4 * q + 7], v.w, a1);
  }
  return a0 + a1;
}

__device__ __forceinline__ void normalise(const MlpW &s, const float f[4], float x[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = (f[k] - s.mu[k]) / s.sd[k];
}

// full forward pass of one sample
__device__ __forceinline__ void mlp_forward(const MlpW &s, const float f[4], float &o0, float &o1) {
  float x[4], h1[MH];
  normalise(s, f, x);
  layer1(s, x, h1);
  o0 = s.b3[0];
  o1 = s.b3[1];
  for (int j = 0; j < MH; ++j) {
    const float h = tanhf(layer2_pre(s, h1, j));
    o0 = fmaf(h, s.w3[2 * j], o0);
    o1 = fmaf(h, s.w3[2 * j + 1], o1);
  }
}

__global__ void __launch_bounds__(TS, 1) k_mlp_grad(const float *__restrict__ W, const float4 *__restrict__ feat,
                                                    const float2 *__restrict__ tgt, const float2 *__restrict__ wt, long long n,
                                                    double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smraw);
  const int tid = threadIdx.x;
  load_weights(S.w, W);
  for (int t = tid; t < kMlpParams + 1; t += TS) S.g[t] = 0.0;
  __syncthreads();
  const long long ntile = (n + TS - 1) / TS;
  for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const long long smp = tile * TS + tid;
    float f[4] = {0.f, 0.f, 0.f, 0.f}, t0 = 0.f, t1 = 0.f, w0 = 0.f, w1 = 0.f;
    if (smp < n) {  // past the end: zero weight, so nothing flows back
      const float4 fv = feat[smp];
      f[0] = fv.x;
      f[1] = fv.y;
      f[2] = fv.z;
      f[3] = fv.w;
      const float2 tv = tgt[smp], wv = wt[smp];
      t0 = tv.x;
      t1 = tv.y;
      w0 = wv.x;
      w1 = wv.y;
    }
    float x[4], h1[MH];
    normalise(S.w, f, x);
    layer1(S.w, x, h1);
    float o0 = S.w.b3[0], o1 = S.w.b3[1];
    for (int j = 0; j < MH; ++j) {
      const float h = tanhf(layer2_pre(S.w, h1, j));
      S.H2[tid * P65 + j] = h;
      o0 = fmaf(h, S.w.w3[2 * j], o0);
      o1 = fmaf(h, S.w.w3[2 * j + 1], o1);
    }
    const float r0 = o0 - t0, r1 = o1 - t1;
    const float e0 = 2.f * w0 * r0, e1 = 2.f * w1 * r1;  // dL/do
    double lsum = (double)w0 * r0 * r0 + (double)w1 * r1 * r1;
    // backward: d2_j = (W3[j] . e) (1 - h2_j^2); d1_i = (sum_j W2[i][j] d2_j) (1 - h1_i^2)
    float d1[MH];
#pragma unroll
    for (int i = 0; i < MH; ++i) d1[i] = 0.f;
    for (int j = 0; j < MH; ++j) {
      const float h = S.H2[tid * P65 + j];
      const float d2 = (S.w.w3[2 * j] * e0 + S.w.w3[2 * j + 1] * e1) * (1.f - h * h);
      S.D2[tid * P68 + j] = d2;
      const float4 *wr = reinterpret_cast<const float4 *>(S.w.w2t + j * MH);
#pragma unroll
      for (int q = 0; q < MH / 4; ++q) {
        const float4 u = wr[q];
        d1[4 * q + 0] = fmaf(u.x, d2, d1[4 * q + 0]);
        d1[4 * q + 1] = fmaf(u.y, d2, d1[4 * q + 1]);
        d1[4 * q + 2] = fmaf(u.z, d2, d1[4 * q + 2]);
        d1[4 * q + 3] = fmaf(u.w, d2, d1[4 * q + 3]);
      }
    }
#pragma unroll
    for (int i = 0; i < MH; ++i) {
      S.D1[tid * P65 + i] = d1[i] * (1.f - h1[i] * h1[i]);
      S.H1[tid * P65 + i] = h1[i];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) S.X[tid * 4 + k] = x[k];
    S.E[tid * 2] = e0;
    S.E[tid * 2 + 1] = e1;
    // loss of the tile
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
      double l = 0.0;
      for (int w = 0; w < TS / 32; ++w) l += S.red[w];
      S.g[kMlpParams] += l;
    }
    // weight gradients of the tile: each entry belongs to one thread
    {
      const int i = tid >> 1, jb = (tid & 1) * 32;  // W2[i][jb .. jb+31]
      float acc[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) acc[q] = 0.f;
      for (int s = 0; s < TS; ++s) {
        const float h = S.H1[s * P65 + i];
        const float4 *dr = reinterpret_cast<const float4 *>(S.D2 + s * P68 + jb);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 d = dr[q];
          acc[4 * q + 0] = fmaf(h, d.x, acc[4 * q + 0]);
          acc[4 * q + 1] = fmaf(h, d.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(h, d.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(h, d.w, acc[4 * q + 3]);
        }
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) S.g[OW2 + i * MH + jb + q] += (double)acc[q];
    }
    {
      const int i = tid >> 1, kb = (tid & 1) * 2;  // W1[kb..kb+1][i]
      const int j = tid >> 1, k = tid & 1;         // W3[j][k]
      float a0 = 0.f, a1 = 0.f, a3 = 0.f, ab = 0.f;
      for (int s = 0; s < TS; ++s) {
        const float d = S.D1[s * P65 + i];
        a0 = fmaf(S.X[s * 4 + kb], d, a0);
        a1 = fmaf(S.X[s * 4 + kb + 1], d, a1);
        a3 = fmaf(S.H2[s * P65 + j], S.E[s * 2 + k], a3);
        ab += tid < MH ? S.D1[s * P65 + tid] : S.D2[s * P68 + (tid - MH)];
      }
      S.g[OW1 + kb * MH + i] += (double)a0;
      S.g[OW1 + (kb + 1) * MH + i] += (double)a1;
      S.g[OW3 + j * 2 + k] += (double)a3;
      if (tid < MH) S.g[OB1 + tid] += (double)ab;
      else S.g[OB2 + tid - MH] += (double)ab;
      if (tid < 2) {
        float e = 0.f;
        for (int s = 0; s < TS; ++s) e += S.E[s * 2 + tid];
        S.g[OB3 + tid] += (double)e;
      }
    }
    __syncthreads();  // the next tile overwrites the activations
  }
  for (int t = tid; t < kMlpParams + 1; t += TS) part[(size_t)blockIdx.x * (kMlpParams + 1) + t] = S.g[t];
}

__global__ void k_mlp_reduce(const double *__restrict__ part, int nblk, double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > kMlpParams) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (kMlpParams + 1) + t];
  out[t] = s;
}

__global__ void k_mlp_adam(double *__restrict__ w64, float *__restrict__ w32, const double *__restrict__ g, double *__restrict__ m,
                           double *__restrict__ v, double lr, double c1, double c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kMlpParams) return;
  const double gt = g[t];
  const double mt = 0.9 * m[t] + 0.1 * gt;
  const double vt = 0.999 * v[t] + 0.001 * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const double w = w64[t] - lr * (mt * c1) / (sqrt(vt * c2) + 1e-8);
  w64[t] = w;
  w32[t] = (float)w;
}

// features of orbital v at internal element e (FP64 arithmetic, rounded to FP32 like the samples)
__device__ __forceinline__ void sample_features(const Geo &g, int e, double tk, double ev, const cplx<double> &c, double nh,
                                                float f[4]) {
  f[0] = (float)log1p(0.5 * g.g2[e] / tk);
  f[1] = (float)ev;
  f[2] = (float)tk;
  f[3] = (float)log(nh * (c.x * c.x + c.y * c.y) + 1e-6);
}

__global__ void __launch_bounds__(128) k_mlp_table(Geo g, const float *__restrict__ W, const cplx<double> *__restrict__ psi,
                                                   const double *__restrict__ tkin, const double *__restrict__ eps, double nh,
                                                   const double *__restrict__ ktpa, int nocc, double *__restrict__ m64,
                                                   float *__restrict__ m32, double *__restrict__ w64) {
  __shared__ __align__(16) MlpW s;
  load_weights(s, W);
  __syncthreads();
  const int v = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ld) return;
  const size_t o = (size_t)v * g.ld + e;
  const double k = ktpa[o];
  double mk = 0.0, wk = 0.0;
  if (e < g.nint) {
    float f[4], o0, o1;
    sample_features(g, e, tkin[v], eps[v], psi[o], nh, f);
    mlp_forward(s, f, o0, o1);
    mk = exp((double)fminf(fmaxf(o0, -8.f), 8.f)) * k;
    wk = (double)o1 * k;
  }
  m64[o] = mk;                               // learned rows [0, nocc)
  m32[o] = (float)mk;
  m64[(size_t)nocc * g.ld + o] = k;          // TPA rows [nocc, 2 nocc) for the fallback
  m32[(size_t)nocc * g.ld + o] = (float)k;
  w64[o] = wk;
}

__global__ void __launch_bounds__(128) k_mlp_predict(const float *__restrict__ W, const float4 *__restrict__ feat, long long n,
                                                     float2 *__restrict__ out) {
  __shared__ __align__(16) MlpW s;
  load_weights(s, W);
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 fv = feat[i];
  const float f[4] = {fv.x, fv.y, fv.z, fv.w};
  float o0, o1;
  mlp_forward(s, f, o0, o1);
  out[i] = make_float2(o0, o1);
}

// sums[0|1|2][v][e] += |x|^2, |K b|^2, Re(conj(K b) x) over the solves of orbital v; solve s of a
// chi0bar block belongs to orbital (s / 2) % nocc and nq / nocc = the perturbation pairs
__global__ void k_mlp_accum(Geo g, const cplx<double> *__restrict__ b, const cplx<double> *__restrict__ x, int ns, int nocc,
                            const double *__restrict__ ktpa, double *__restrict__ sums) {
  const int v = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.nint) return;
  const double k = ktpa[(size_t)v * g.ld + e];
  double ex = 0.0, ek = 0.0, ck = 0.0;
  const int npair = ns / (2 * nocc);
  for (int q = 0; q < npair; ++q)
    for (int h = 0; h < 2; ++h) {
      const size_t row = (size_t)2 * (q * nocc + v) + h;
      const cplx<double> bv = b[row * g.ld + e], xv = x[row * g.ld + e];
      const double kbx = k * bv.x, kby = k * bv.y;
      ex += xv.x * xv.x + xv.y * xv.y;
      ek += kbx * kbx + kby * kby;
      ck += kbx * xv.x + kby * xv.y;
    }
  const size_t o = (size_t)v * g.ld + e, plane = (size_t)nocc * g.ld;
  sums[o] += ex;
  sums[plane + o] += ek;
  sums[2 * plane + o] += ck;
}

// one sample per (v, half-sphere index i): features, targets, raw weights (counted for G and -G)
__global__ void k_mlp_samples(Geo g, const int *__restrict__ emap, int npw_h, int nocc, const double *__restrict__ sums,
                              const cplx<double> *__restrict__ psi, const double *__restrict__ tkin, const double *__restrict__ eps,
                              float4 *__restrict__ feat, float2 *__restrict__ tgt, double *__restrict__ wraw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nocc * npw_h) return;
  const int v = (int)(t / npw_h), i = (int)(t % npw_h);
  const int e = emap[i];
  const size_t o = (size_t)v * g.ld + e, plane = (size_t)nocc * g.ld;
  float f[4];
  sample_features(g, e, tkin[v], eps[v], psi[o], (double)npw_h, f);
  feat[t] = make_float4(f[0], f[1], f[2], f[3]);
  const double ex = sums[o], ek = sums[plane + o], ck = sums[2 * plane + o];
  const double mult = i == 0 ? 1.0 : 2.0;
  const bool ok = ek > 0.0;
  tgt[t] = make_float2(ok ? (float)(0.5 * (log(ex + 1e-300) - log(ek))) : 0.f, ok ? (float)(ck / ek) : 0.f);
  wraw[2 * t] = ok ? (ex + ek) * mult : 0.0;
  wraw[2 * t + 1] = ok ? ek * mult : 0.0;
}

// column sums of wraw[n][2] by one block in a fixed order
__global__ void k_mlp_wsum(const double *__restrict__ wraw, long long n, double *__restrict__ out) {
  __shared__ double r0[256], r1[256];
  double a0 = 0.0, a1 = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    a0 += wraw[2 * t];
    a1 += wraw[2 * t + 1];
  }
  r0[threadIdx.x] = a0;
  r1[threadIdx.x] = a1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r0[threadIdx.x] += r0[threadIdx.x + s];
      r1[threadIdx.x] += r1[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r0[0];
    out[1] = r1[0];
  }
}

__global__ void k_mlp_wnorm(const double *__restrict__ wraw, long long n, const double *__restrict__ sum, float2 *__restrict__ wt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double s0 = sum[0] > 0.0 ? sum[0] : 1.0, s1 = sum[1] > 0.0 ? sum[1] : 1.0;
  wt[t] = make_float2((float)(wraw[2 * t] / s0), (float)(wraw[2 * t + 1] / s1));
}

__global__ void k_first_iterate(Geo g, cplx<double> *__restrict__ x, const cplx<double> *__restrict__ b, const double *__restrict__ w,
                                const int *__restrict__ vidx, int n) {
  const size_t tot = (size_t)n * g.ld;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / g.ld), e = (int)(t % g.ld);
    const double k = w[(size_t)vidx[s] * g.ld + e];
    const cplx<double> bv = b[t];
    x[t] = mkc<double>(k * bv.x, k * bv.y);
  }
}

int grad_blocks(long long n) {
  const long long ntile = (n + TS - 1) / TS;
  return (int)std::max<long long>(1, std::min<long long>(ntile, 152));
}

}  // namespace

size_t mlp_grad_smem() { return sizeof(TrainSmem); }

void set_mlp_limits() {
  raise_smem_limit(k_mlp_grad, (size_t)((int)sizeof(TrainSmem)));
}

int mlp_grad_blocks(long long n) { return grad_blocks(n); }

void launch_mlp_grad(const float *W, const float *feat, const float *tgt, const float *wt, long long n, double *part, double *out,
                     cudaStream_t st) {
  const int nb = grad_blocks(n);
  launch("mlp_grad", 32, k_mlp_grad, dim3(nb), dim3(TS), sizeof(TrainSmem), st, W, reinterpret_cast<const float4 *>(feat),
         reinterpret_cast<const float2 *>(tgt), reinterpret_cast<const float2 *>(wt), n, part);
  WDF_CUDA_TRY(cudaGetLastError());
  launch("mlp_reduce", 64, k_mlp_reduce, dim3((kMlpParams + 1 + 255) / 256), dim3(256), 0, st, (const double *)part, nb, out);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_mlp_adam(double *w64, float *w32, const double *grad, double *m, double *v, int t, double lr, cudaStream_t st) {
  const double c1 = 1.0 / (1.0 - std::pow(0.9, t)), c2 = 1.0 / (1.0 - std::pow(0.999, t));
  launch("mlp_adam", 64, k_mlp_adam, dim3((kMlpParams + 255) / 256), dim3(256), 0, st, w64, w32, grad, m, v, lr, c1, c2);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_mlp_table(const Geo &g, const float *W, const cplx<double> *psi, const double *tkin, const double *eps, int npw_h,
                      const double *ktpa, int nocc, double *m64, float *m32, double *w64, cudaStream_t st) {
  launch("mlp_table", 32, k_mlp_table, dim3((g.ld + 127) / 128, nocc), dim3(128), 0, st, g, W, psi, tkin, eps, (double)npw_h, ktpa,
         nocc, m64, m32, w64);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_mlp_predict(const float *W, const float *feat, long long n, float *out, cudaStream_t st) {
  if (n <= 0) return;
  launch("mlp_predict", 32, k_mlp_predict, dim3((unsigned)((n + 127) / 128)), dim3(128), 0, st, W,
         reinterpret_cast<const float4 *>(feat), n, reinterpret_cast<float2 *>(out));
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_first_iterate(const Geo &g, cplx<double> *x, const cplx<double> *b, const double *w, const int *vidx, int n,
                          cudaStream_t st) {
  if (n <= 0) return;
  launch("mlp_table", 64, k_first_iterate, dim3(std::min(4096, (int)(((size_t)n * g.ld + 255) / 256))), dim3(256), 0, st, g, x, b, w,
         vidx, n);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_mlp_accum(const Geo &g, const cplx<double> *b, const cplx<double> *x, int ns, int nocc, const double *ktpa, double *sums,
                      cudaStream_t st) {
  if (ns <= 0) return;
  launch("mlp_accum", 64, k_mlp_accum, dim3((g.nint + 255) / 256, nocc), dim3(256), 0, st, g, b, x, ns, nocc, ktpa, sums);
  WDF_CUDA_TRY(cudaGetLastError());
}

void launch_mlp_samples(const Geo &g, const int *emap, int npw_h, int nocc, const double *sums, const cplx<double> *psi,
                        const double *tkin, const double *eps, float *feat, float *tgt, float *wt, double *wraw, double *wsum,
                        cudaStream_t st) {
  const long long n = (long long)nocc * npw_h;
  if (n <= 0) return;
  const unsigned nb = (unsigned)((n + 255) / 256);
  launch("mlp_samples", 64, k_mlp_samples, dim3(nb), dim3(256), 0, st, g, emap, npw_h, nocc, sums, psi, tkin, eps,
         reinterpret_cast<float4 *>(feat), reinterpret_cast<float2 *>(tgt), wraw);
  WDF_CUDA_TRY(cudaGetLastError());
  launch("mlp_samples", 64, k_mlp_wsum, dim3(1), dim3(256), 0, st, (const double *)wraw, n, wsum);
  WDF_CUDA_TRY(cudaGetLastError());
  launch("mlp_samples", 64, k_mlp_wnorm, dim3(nb), dim3(256), 0, st, (const double *)wraw, n, (const double *)wsum,
         reinterpret_cast<float2 *>(wt));
  WDF_CUDA_TRY(cudaGetLastError());
}

}  // namespace wdf

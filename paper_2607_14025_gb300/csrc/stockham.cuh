// Compile-time Stockham FFT passes shared by the plane kernels and the n3 transforms.
//
// A length-N transform runs its radices 8, 4, 5, 3, 2 (largest first; the forward transform in
// the reverse order). Pass (radix R, stride Ls): butterfly j reads elements j + r N / R of its
// line, multiplies element r by w^(r k / (Ls R)) with k = j mod Ls (w = exp(+2 pi i / N) for the
// inverse, the conjugate for the forward transform), does an R-point DFT in registers and writes
// element (j / Ls) Ls R + k + r Ls. Input and output are in natural order (no digit reversal).
#pragma once

#include "fft.cuh"
#include "kernels.cuh"

namespace wdf {

// radices: 8 first, then 4, 5, 3, 2
__host__ __device__ constexpr int rad_at(int n, int p) {
  int m = n;
  int idx = 0;
  const int pr[5] = {8, 4, 5, 3, 2};
  for (int i = 0; i < 5; ++i) {
    while (m % pr[i] == 0) {
      if (idx == p) return pr[i];
      m /= pr[i];
      ++idx;
    }
  }
  return 1;
}
__host__ __device__ constexpr int nrad(int n) {
  int c = 0;
  while (rad_at(n, c) > 1) ++c;
  return c;
}
__host__ __device__ constexpr int ls_at(int n, int p) {  // product of the radices before pass p
  int l = 1;
  for (int i = 0; i < p; ++i) l *= rad_at(n, i);
  return l;
}
// forward passes run the radices in reverse order
__host__ __device__ constexpr int frad_at(int n, int p) { return rad_at(n, nrad(n) - 1 - p); }
__host__ __device__ constexpr int fls_at(int n, int p) {
  int l = 1;
  for (int i = 0; i < p; ++i) l *= frad_at(n, i);
  return l;
}
__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

// double-float 8-point DFT with unnormalised sums inside its two 4-point halves (and inside the
// w8 products), renormalised once at the outputs: the same operations as the generic form below
// in the same order, about 100 FP32 operations fewer; float32 emulation against the exact DFT
// gives 8.9e-15 relative error against 6.9e-15 for renormalising every sum
template <int SG> __device__ __forceinline__ void dft8_df_lazy(cplx<df64> *v) {
  typedef cplx<df64> C;
  auto ladd = [](C a, C b) { return mkc<df64>(df_add_lazy(a.x, b.x), df_add_lazy(a.y, b.y)); };
  auto lsub = [](C a, C b) { return mkc<df64>(df_add_lazy(a.x, -b.x), df_add_lazy(a.y, -b.y)); };
  auto rad4 = [&](C x0, C x1, C x2, C x3, C(&y)[4]) {
    const C a = ladd(x0, x2), b = lsub(x0, x2), c = ladd(x1, x3), d = cimul_unit<SG, df64>(lsub(x1, x3));
    y[0] = ladd(a, c);
    y[1] = ladd(b, d);
    y[2] = lsub(a, c);
    y[3] = lsub(b, d);
  };
  C e[4], o[4];
  rad4(v[0], v[2], v[4], v[6], e);
  rad4(v[1], v[3], v[5], v[7], o);
  const df64 h = df64(0.70710678118654752440);
  // o1 (1 + SG i)/sqrt2, o2 SG i, o3 (-1 + SG i)/sqrt2
  const C o1 = SG > 0 ? mkc<df64>(h * df_add_lazy(o[1].x, -o[1].y), h * df_add_lazy(o[1].y, o[1].x))
                      : mkc<df64>(h * df_add_lazy(o[1].x, o[1].y), h * df_add_lazy(o[1].y, -o[1].x));
  const C o2 = cimul_unit<SG, df64>(o[2]);
  const C o3 = SG > 0 ? mkc<df64>(h * df_add_lazy(-o[3].x, -o[3].y), h * df_add_lazy(-o[3].y, o[3].x))
                      : mkc<df64>(h * df_add_lazy(o[3].y, -o[3].x), h * df_add_lazy(-o[3].y, -o[3].x));
  const C oo[4] = {o[0], o1, o2, o3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const C s = ladd(e[k], oo[k]), d = lsub(e[k], oo[k]);
    v[k] = mkc<df64>(df_norm(s.x), df_norm(s.y));
    v[k + 4] = mkc<df64>(df_norm(d.x), df_norm(d.y));
  }
}

// modular inverse of a modulo m (a and m coprime, small): the smallest x >= 1 with a x = 1 mod m
__host__ __device__ constexpr int inv_mod(int a, int m) {
  int x = 1;
  while ((a * x) % m != 1) ++x;
  return x;
}

// R = A B point DFT with A and B coprime by the prime-factor (Good-Thomas) map: input n =
// (B n1 + A n2) mod R, output k = (B (B^-1 mod A) k1 + A (A^-1 mod B) k2) mod R, so that
// w_R^(n k) = w_A^(n1 k1) w_B^(n2 k2) and no twiddle factors are needed.
template <typename T, int A, int B, int SG>
__device__ __forceinline__ void dft_pfa(cplx<T> *v) {
  constexpr int R = A * B;
  constexpr int cA = B * inv_mod(B % A, A), cB = A * inv_mod(A % B, B);
  cplx<T> a[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2)
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) a[n2][n1] = v[(B * n1 + A * n2) % R];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) small_dft<T, SG>(a[n2], A);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    cplx<T> b[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) b[n2] = a[n2][k1];
    small_dft<T, SG>(b, B);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[(cA * k1 + cB * k2) % R] = b[k2];
  }
}

template <typename T, int R, int SG>
__device__ __forceinline__ void dft_reg(cplx<T> *v) {
  if constexpr (std::is_same<T, df64>::value && R == 8) {
    dft8_df_lazy<SG>(v);
    return;
  }
  if constexpr (R == 6) {
    dft_pfa<T, 3, 2, SG>(v);
    return;
  }
  if constexpr (R == 10) {
    dft_pfa<T, 5, 2, SG>(v);
    return;
  }
  if constexpr (R == 12) {
    dft_pfa<T, 3, 4, SG>(v);
    return;
  }
  if (R == 8) {
    // radix-2 split into two 4-point DFTs, combined with w8^k = exp(SG 2 pi i k / 8)
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    small_dft<T, SG>(e, 4);
    small_dft<T, SG>(o, 4);
    const T h = (T)0.70710678118654752440;
    // o1 (1 + SG i)/sqrt2, o2 SG i, o3 (-1 + SG i)/sqrt2
    const cplx<T> o1 = SG > 0 ? mkc<T>(h * (o[1].x - o[1].y), h * (o[1].y + o[1].x)) : mkc<T>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    const cplx<T> o2 = cimul_unit<SG, T>(o[2]);
    const cplx<T> o3 = SG > 0 ? mkc<T>(h * (-o[3].x - o[3].y), h * (-o[3].y + o[3].x)) : mkc<T>(h * (o[3].y - o[3].x), h * (-o[3].y - o[3].x));
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], o1);
    v[5] = csub<T>(e[1], o1);
    v[2] = cadd<T>(e[2], o2);
    v[6] = csub<T>(e[2], o2);
    v[3] = cadd<T>(e[3], o3);
    v[7] = csub<T>(e[3], o3);
  } else {
    small_dft<T, SG>(v, R);
  }
}

// One pass over NL lines of length N stored at sm[l * PITCH + t], THREADS threads.
template <typename T, int N, int P, int SIGN, int NL, int PITCH, int THREADS>
__device__ __forceinline__ void zline_pass(cplx<T> *sm, const cplx<T> *tw) {
  constexpr int R = SIGN > 0 ? rad_at(N, P) : frad_at(N, P);
  constexpr int LS = SIGN > 0 ? ls_at(N, P) : fls_at(N, P);
  constexpr int TASKS = NL * (N / R);
  constexpr int TPT = cdiv(TASKS, THREADS);
  cplx<T> v[TPT][R];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + u * THREADS;
    if (TASKS % THREADS == 0 || t < TASKS) {
      const int l = t % NL, j = t / NL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u][r] = sm[l * PITCH + j + r * (N / R)];
      if constexpr (LS > 1) {
        const int k = j % LS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const cplx<T> w = tw[(r * k * (N / (LS * R))) % N];
          v[u][r] = (SIGN > 0) ? cmul<T>(v[u][r], w) : cmulc<T>(v[u][r], w);
        }
      }
      dft_reg<T, R, SIGN>(v[u]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = threadIdx.x + u * THREADS;
    if (TASKS % THREADS == 0 || t < TASKS) {
      const int l = t % NL, j = t / NL;
      const int k = j % LS, o = (j / LS) * LS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[l * PITCH + o + r * LS] = v[u][r];
    }
  }
  __syncthreads();
}

template <typename T, int N, int SIGN, int NL, int PITCH, int THREADS, int P = 0>
__device__ __forceinline__ void zlines_fft(cplx<T> *sm, const cplx<T> *tw) {
  if constexpr (P < nrad(N)) {
    zline_pass<T, N, P, SIGN, NL, PITCH, THREADS>(sm, tw);
    zlines_fft<T, N, SIGN, NL, PITCH, THREADS, P + 1>(sm, tw);
  }
}

}  // namespace wdf

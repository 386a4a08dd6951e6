// Shared-memory FFT building blocks: batched 1-D transforms of lines held in shared memory.
//
// Both directions run in place with no second buffer and no permutation pass:
//  * inverse (sign +, G -> r): decimation in time, input in digit-reversed order, output natural;
//  * forward (sign -, r -> G): decimation in frequency, input natural, output digit-reversed.
// For a length n = r_1 r_2 ... r_k (stages in this order for the inverse), the digit-reversed
// position of index v is pos(v) = (v mod r_k) n/r_k + pos'(v div r_k) with pos' the same map for
// the first k-1 radices; the forward transform runs the stages in reverse order and leaves
// frequency v at pos(v). Callers therefore scatter spectral data to pos() before an inverse
// transform and gather from pos() after a forward one.
//
// A stage of radix r on blocks of length Lb = r Lj:
//  inverse: for each block and k1 < Lj, inputs at k1 + Lj s (s < r) are multiplied by
//           w_Lb^(s k1) and combined by an r-point DFT into the same positions;
//  forward: for each block and n1 < M = Lb/r, inputs at n1 + M s are combined by an r-point DFT
//           and output s is multiplied by w_Lb^(-n1 s).
// Twiddles come from a table tw[t] = exp(2 pi i t / n) (FP64-accurate, from the host).
#pragma once

#include "common.cuh"

namespace wdf {

// a times SG i for SG = +1 or -1: a swap and a sign change, no multiplication (a double-float
// multiply by +-1 would cost seven FP32 operations and the compiler cannot drop it)
template <int SG, typename T> __device__ __forceinline__ cplx<T> cimul_unit(cplx<T> a) {
  return SG > 0 ? mkc<T>(-a.y, a.x) : mkc<T>(a.y, -a.x);
}

// r-point DFT in registers, X_k = sum_s x_s exp(SG 2 pi i s k / r), r in {2, 3, 4, 5}, SG = +-1.
// Constants are cos and sin of 2 pi / 5, 4 pi / 5 and sqrt(3)/2.
template <typename T, int SG>
__device__ __forceinline__ void small_dft(cplx<T> *x, int r) {
  if (r == 4) {
    cplx<T> a = cadd<T>(x[0], x[2]), b = csub<T>(x[0], x[2]);
    cplx<T> c = cadd<T>(x[1], x[3]), d = cimul_unit<SG, T>(csub<T>(x[1], x[3]));
    x[0] = cadd<T>(a, c);
    x[1] = cadd<T>(b, d);
    x[2] = csub<T>(a, c);
    x[3] = csub<T>(b, d);
  } else if (r == 2) {
    cplx<T> a = x[0];
    x[0] = cadd<T>(a, x[1]);
    x[1] = csub<T>(a, x[1]);
  } else if (r == 3) {
    const T s3 = (T)0.86602540378443864676;
    cplx<T> t = cadd<T>(x[1], x[2]);
    cplx<T> u = mkc<T>(x[0].x - (T)0.5 * t.x, x[0].y - (T)0.5 * t.y);
    cplx<T> v = cimul<T>(csub<T>(x[1], x[2]), SG > 0 ? s3 : -s3);
    x[0] = cadd<T>(x[0], t);
    x[1] = cadd<T>(u, v);
    x[2] = csub<T>(u, v);
  } else {  // r == 5
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    cplx<T> a1 = cadd<T>(x[1], x[4]), a2 = cadd<T>(x[2], x[3]);
    cplx<T> b1 = csub<T>(x[1], x[4]), b2 = csub<T>(x[2], x[3]);
    cplx<T> p = mkc<T>(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
    cplx<T> q = mkc<T>(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
    cplx<T> u = cimul_unit<SG, T>(mkc<T>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    cplx<T> w = cimul_unit<SG, T>(mkc<T>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    x[0] = cadd<T>(x[0], cadd<T>(a1, a2));
    x[1] = cadd<T>(p, u);
    x[4] = csub<T>(p, u);
    x[2] = cadd<T>(q, w);
    x[3] = csub<T>(q, w);
  }
}

// Transform nlines lines held in shared memory. Line l starts at base(l) = line_base[l] (if
// line_base != nullptr) or l * line_pitch; element t of a line sits at base(l) + t * es.
// INVERSE = true: decimation-in-time inverse transform (digit-reversed in, natural out).
// INVERSE = false: decimation-in-frequency forward transform (natural in, digit-reversed out).
// Every thread of the block must call this (it synchronises between stages and at the end).
template <typename T, bool INVERSE>
__device__ void fft_lines(cplx<T> *sm, int nlines, const int *line_base, int line_pitch, int es,
                          const Plan1D &P, const cplx<T> *tw) {
  const int n = P.n;
  for (int st = 0; st < P.nst; ++st) {
    const int j = INVERSE ? st : (P.nst - 1 - st);
    const int r = P.r[j];
    const int Lj = P.L[j];
    const int Lb = P.L[j + 1];
    const int tstep = n / Lb;
    const int nb = n / r;
    const int total = nlines * nb;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
      const int l = it % nlines;
      const int bi = it / nlines;
      const int base = line_base ? line_base[l] : l * line_pitch;
      const int b = bi / Lj;
      const int k1 = bi - b * Lj;
      const int p0 = b * Lb + k1;
      cplx<T> x[5];
      // loops run to the largest radix and test s < r so that x[] stays in registers
      if (INVERSE) {
        x[0] = sm[base + p0 * es];
#pragma unroll
        for (int s = 1; s < 5; ++s)
          if (s < r) x[s] = cmul<T>(sm[base + (p0 + s * Lj) * es], tw[s * k1 * tstep]);
        small_dft<T, 1>(x, r);
#pragma unroll
        for (int s = 0; s < 5; ++s)
          if (s < r) sm[base + (p0 + s * Lj) * es] = x[s];
      } else {
#pragma unroll
        for (int s = 0; s < 5; ++s)
          if (s < r) x[s] = sm[base + (p0 + s * Lj) * es];
        small_dft<T, -1>(x, r);
        sm[base + p0 * es] = x[0];
#pragma unroll
        for (int s = 1; s < 5; ++s)
          if (s < r) sm[base + (p0 + s * Lj) * es] = cmulc<T>(x[s], tw[s * k1 * tstep]);
      }
    }
    __syncthreads();
  }
}

}  // namespace wdf

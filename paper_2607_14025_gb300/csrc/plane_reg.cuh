// Whole 64-or-fewer-point FP32 lines in registers (N = 8 R2, R2 in {3, 4, 5, 8}): a four-step
// DFT with static register indices (8-point DFTs over stride-R2 subsequences, twiddles, R2-point
// DFTs over consecutive slots). The inverse takes natural order and leaves X[k1 + 8 k2] in slot
// k2 + R2 k1; the forward transform takes exactly that permuted order and returns natural order,
// so an inverse, a pointwise product and a forward transform of one line never leave registers.
#pragma once

#include "fft.cuh"
#include "stockham.cuh"

namespace wdf {

template <int N>
__device__ __forceinline__ void line_inverse(float2 (&x)[N], const float2 *tw) {
  constexpr int R2 = N / 8;
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    float2 a[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) a[n1] = x[n2 + R2 * n1];
    dft_reg<float, 8, 1>(a);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) x[n2 + R2 * k1] = (n2 * k1 == 0) ? a[k1] : cmul<float>(a[k1], tw[n2 * k1]);
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = x[n2 + R2 * k1];
    dft_reg<float, R2, 1>(b);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k2 + R2 * k1] = b[k2];
  }
}

template <int N>
__device__ __forceinline__ void line_forward(float2 (&x)[N], const float2 *tw) {
  constexpr int R2 = N / 8;
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 b[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) b[k2] = x[k2 + R2 * k1];
    dft_reg<float, R2, -1>(b);
#pragma unroll
    for (int q2 = 0; q2 < R2; ++q2) x[q2 + R2 * k1] = (k1 * q2 == 0) ? b[q2] : cmulc<float>(b[q2], tw[k1 * q2]);
  }
#pragma unroll
  for (int q2 = 0; q2 < R2; ++q2) {
    float2 a[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) a[k1] = x[q2 + R2 * k1];
    dft_reg<float, 8, -1>(a);
#pragma unroll
    for (int q1 = 0; q1 < 8; ++q1) x[q2 + R2 * q1] = a[q1];
  }
}

// natural index held by slot s after line_inverse
template <int N> __device__ __forceinline__ constexpr int perm_index(int s) { return s / (N / 8) + 8 * (s % (N / 8)); }

}  // namespace wdf

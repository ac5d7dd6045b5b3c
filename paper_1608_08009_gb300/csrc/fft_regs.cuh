// In-register radix-2 FFT of one pencil, fully unrolled (N = 16, 32, 64).
//
// Used for every 1D pass of the 3D transforms of the fast spectral collision operator
// (arxiv 1608.08009, Sec. 3.3, Eqs. FU/FC; Sec. 4.2: one forward transform of f and, per
// direction, the inverse transforms that dominate the cost).  The twiddles
// exp(2 pi i m / 64) come from constant memory, filled once per device by the host with
// the host libm cos/sin in float64 (and rounded to float32 for the float32 path).
#pragma once

#include <cuda_runtime.h>

namespace boltz {

// Defined here; this header is included by exactly one translation unit (collide.cu).
__constant__ double c_twc64[64];
__constant__ double c_tws64[64];
__constant__ float c_twc32[64];
__constant__ float c_tws32[64];

template <typename T> __device__ __forceinline__ T tw_cos(int m);
template <typename T> __device__ __forceinline__ T tw_sin(int m);
template <> __device__ __forceinline__ double tw_cos<double>(int m) { return c_twc64[m]; }
template <> __device__ __forceinline__ double tw_sin<double>(int m) { return c_tws64[m]; }
template <> __device__ __forceinline__ float tw_cos<float>(int m) { return c_twc32[m]; }
template <> __device__ __forceinline__ float tw_sin<float>(int m) { return c_tws32[m]; }

template <int N>
__host__ __device__ constexpr int bit_reverse(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// x_k <- sum_j x_j exp(SIGN 2 pi i j k / N); no scaling.  SIGN = -1 forward, +1 inverse.
template <int N, int SIGN, typename T>
__device__ __forceinline__ void fft_regs(T (&xr)[N], T (&xi)[N]) {
  static_assert((N & (N - 1)) == 0 && N <= 64, "power of two up to 64");
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bit_reverse<N>(i);
    if (j > i) {
      T t = xr[i]; xr[i] = xr[j]; xr[j] = t;
      t = xi[i]; xi[i] = xi[j]; xi[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
    const int stride = 64 / len;
#pragma unroll
    for (int s = 0; s < N; s += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int m = k * stride;  // twiddle exp(SIGN 2 pi i m / 64)
        const T br = xr[s + k + half], bi = xi[s + k + half];
        T tr, ti;
        if (m == 0) {
          tr = br; ti = bi;
        } else if (m == 16) {  // exp(SIGN i pi / 2) = SIGN i
          tr = (SIGN > 0) ? -bi : bi;
          ti = (SIGN > 0) ? br : -br;
        } else {
          const T c = tw_cos<T>(m);
          const T sn = (SIGN > 0) ? tw_sin<T>(m) : -tw_sin<T>(m);
          tr = br * c - bi * sn;
          ti = br * sn + bi * c;
        }
        xr[s + k + half] = xr[s + k] - tr;
        xi[s + k + half] = xi[s + k] - ti;
        xr[s + k] = xr[s + k] + tr;
        xi[s + k] = xi[s + k] + ti;
      }
    }
  }
}

}  // namespace boltz

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

// Bit-reversal permutation of 0..N-1 as a compile-time table, so that the register
// arrays below are only ever indexed by constants (otherwise they are placed in local
// memory).
template <int N>
struct BitReverse {
  int v[N];
  constexpr BitReverse() : v() {
    for (int i = 0; i < N; ++i) {
      int r = 0, x = i;
      for (int b = 1; b < N; b <<= 1) {
        r = (r << 1) | (x & 1);
        x >>= 1;
      }
      v[i] = r;
    }
  }
};

// One radix-2 decimation-in-time stage of butterflies of span LEN, then the next stage.
// LEN is a template parameter so every loop has compile-time bounds and unrolls fully:
// the register arrays are only ever indexed by constants.
template <int N, int SIGN, int LEN, typename T>
__device__ __forceinline__ void fft_stage(T (&xr)[N], T (&xi)[N]) {
  constexpr int half = LEN / 2;
  constexpr int stride = 64 / LEN;
#pragma unroll
  for (int s = 0; s < N; s += LEN) {
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
  if constexpr (LEN < N) fft_stage<N, SIGN, 2 * LEN>(xr, xi);
}

// x_k <- sum_j x_j exp(SIGN 2 pi i j k / N); no scaling.  SIGN = -1 forward, +1 inverse.
template <int N, int SIGN, typename T>
__device__ __forceinline__ void fft_regs(T (&xr)[N], T (&xi)[N]) {
  static_assert((N & (N - 1)) == 0 && N >= 2 && N <= 64, "power of two up to 64");
  constexpr BitReverse<N> rev{};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = rev.v[i];
    if (j > i) {
      T t = xr[i]; xr[i] = xr[j]; xr[j] = t;
      t = xi[i]; xi[i] = xi[j]; xi[j] = t;
    }
  }
  fft_stage<N, SIGN, 2>(xr, xi);
}

}  // namespace boltz

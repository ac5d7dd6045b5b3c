// In-register FFT of one pencil, fully unrolled: N = 2^k (radix-4/2) or N = 3 * 2^k
// (one radix-3 decimation over three power-of-two sub-transforms), N <= 64.
//
// Used for every 1D pass of the 3D transforms of the fast spectral collision operator
// (arxiv 1608.08009, Sec. 3.3, Eqs. FU/FC; Sec. 4.2: one forward transform of f and, per
// direction, the inverse transforms that dominate the cost).  The twiddles
// exp(2 pi i m / 192) (192 = lcm of every stage length used) come from constant memory,
// filled once per device by the host with the host libm cos/sin in float64 (and rounded
// to float32 for the float32 path).
//
// The radix-4 stages use the factored twiddles of Linzer and Feig (IBM J. Res. Dev. 37,
// 1993): w = lam i^e (1 + i mu) with |mu| <= 1, the quarter turn i^e a renaming and the
// real factor lam carried into the following additions as fused multiply-adds.  A radix-4
// butterfly with three non-trivial twiddles then costs 22 fused multiply-adds instead of
// 12 multiplications/multiply-adds and 16 additions.
#pragma once

#include <cuda_runtime.h>

#include "twiddles.h"

namespace boltz {

// One copy per translation unit that includes this header (internal linkage); the host
// fills every unit's copy through that unit's upload function.
static __constant__ double c_twc64[kTw];
static __constant__ double c_tws64[kTw];
static __constant__ float c_twc32[kTw];
static __constant__ float c_tws32[kTw];
// Factored twiddles, theta = 2 pi m / 192 (m not a multiple of 48): where
// |cos theta| >= |sin theta|, lam = cos theta and mu = tan theta; otherwise
// lam = sin theta and mu = cot theta.  rho[m] = lam[3m mod 192] / lam[m] (the radix-4
// pair w, w^3).
static __constant__ double c_twl64[kTw];
static __constant__ double c_twm64[kTw];
static __constant__ double c_twr64[kTw];
static __constant__ float c_twl32[kTw];
static __constant__ float c_twm32[kTw];
static __constant__ float c_twr32[kTw];

template <typename T> __device__ __forceinline__ T tw_cos(int m);
template <typename T> __device__ __forceinline__ T tw_sin(int m);
template <> __device__ __forceinline__ double tw_cos<double>(int m) { return c_twc64[m]; }
template <> __device__ __forceinline__ double tw_sin<double>(int m) { return c_tws64[m]; }
template <> __device__ __forceinline__ float tw_cos<float>(int m) { return c_twc32[m]; }
template <> __device__ __forceinline__ float tw_sin<float>(int m) { return c_tws32[m]; }
template <typename T> __device__ __forceinline__ T tw_lam(int m);
template <typename T> __device__ __forceinline__ T tw_mu(int m);
template <typename T> __device__ __forceinline__ T tw_rho(int m);
template <> __device__ __forceinline__ double tw_lam<double>(int m) { return c_twl64[m]; }
template <> __device__ __forceinline__ double tw_mu<double>(int m) { return c_twm64[m]; }
template <> __device__ __forceinline__ double tw_rho<double>(int m) { return c_twr64[m]; }
template <> __device__ __forceinline__ float tw_lam<float>(int m) { return c_twl32[m]; }
template <> __device__ __forceinline__ float tw_mu<float>(int m) { return c_twm32[m]; }
template <> __device__ __forceinline__ float tw_rho<float>(int m) { return c_twr32[m]; }

// x i^e (e taken mod 4): a renaming with sign changes, no arithmetic.
template <typename T>
__device__ __forceinline__ void qturn(int e, T xr, T xi, T& yr, T& yi) {
  e &= 3;
  if (e == 0) {
    yr = xr; yi = xi;
  } else if (e == 1) {
    yr = -xi; yi = xr;
  } else if (e == 2) {
    yr = -xr; yi = -xi;
  } else {
    yr = xi; yi = -xr;
  }
}

// exp(SIGN 2 pi i m / 192) x = lam i^e u with u = x (1 + i mu): returns u already turned
// by i^e and lam (1 for quarter turns, where u is x turned).  m is a compile-time constant
// after unrolling, so the branches fold.
template <int SIGN, typename T>
__device__ __forceinline__ T tw_factor(int m, T xr, T xi, T& ur, T& ui) {
  m %= kTw;
  constexpr int Q = kTw / 4;
  if (m % Q == 0) {
    qturn<T>(SIGN * (m / Q), xr, xi, ur, ui);
    return T(1);
  }
  const int r = m % (kTw / 2);
  const bool cos_form = (r <= kTw / 8) || (r >= 3 * kTw / 8);
  // cos form: w = cos (1 + i SIGN tan); sin form: w = (SIGN i) sin (1 - i SIGN cot)
  const T mu = (cos_form ? T(SIGN) : T(-SIGN)) * tw_mu<T>(m);
  const T vr = xr - mu * xi, vi = xi + mu * xr;
  qturn<T>(cos_form ? 0 : SIGN, vr, vi, ur, ui);
  return tw_lam<T>(m);
}

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

// Complex multiply of (br, bi) by the twiddle exp(SIGN 2 pi i m / 192), m a compile-time
// constant after unrolling (multiples of a quarter turn need no multiplication); used by
// the radix-2 and radix-3 combinations.
template <int SIGN, typename T>
__device__ __forceinline__ void twiddle(int m, T br, T bi, T& tr, T& ti) {
  m %= kTw;
  if (m == 0) {
    tr = br; ti = bi;
  } else if (m == kTw / 4) {  // SIGN i
    tr = (SIGN > 0) ? -bi : bi;
    ti = (SIGN > 0) ? br : -br;
  } else if (m == kTw / 2) {  // -1
    tr = -br; ti = -bi;
  } else if (m == 3 * kTw / 4) {  // -SIGN i
    tr = (SIGN > 0) ? bi : -bi;
    ti = (SIGN > 0) ? -br : br;
  } else {
    const T c = tw_cos<T>(m);
    const T sn = (SIGN > 0) ? tw_sin<T>(m) : -tw_sin<T>(m);
    tr = br * c - bi * sn;
    ti = br * sn + bi * c;
  }
}

// Decimation-in-time stages on bit-reversed input.  SPAN is the length of the
// sub-transforms already formed; a radix-4 stage merges four of them (span 4 SPAN; the
// twiddles w^2, w, w^3 of the four points in factored form, the inner factor SIGN i a
// swap), a radix-2 stage two of them (plain complex multiply).  Spans are template
// parameters so every loop has compile-time bounds and unrolls fully: register indices
// are all constants.
template <int N, int SIGN, int SPAN, typename T>
__device__ __forceinline__ void fft_stages(T (&xr)[N], T (&xi)[N]) {
  if constexpr (SPAN < N) {
    if constexpr (4 * SPAN <= N) {
      constexpr int L = 4 * SPAN;
      constexpr int stride = kTw / L;  // exp(SIGN 2 pi i k / L) = twiddle index k * stride
#pragma unroll
      for (int s = 0; s < N; s += L) {
#pragma unroll
        for (int k = 0; k < SPAN; ++k) {
          const int i0 = s + k, i1 = i0 + SPAN, i2 = i1 + SPAN, i3 = i2 + SPAN;
          const int mB = (k * stride) % kTw;  // w; w^2 at 2 mB, w^3 at 3 mB
          // t0, t1 = x0 +- w^2 x1 with w^2 x1 = lamA u1
          T u1r, u1i;
          const T lamA = tw_factor<SIGN>(2 * mB, xr[i1], xi[i1], u1r, u1i);
          T t0r, t0i, t1r, t1i;
          if ((2 * mB) % (kTw / 4) == 0) {
            t0r = xr[i0] + u1r; t0i = xi[i0] + u1i;
            t1r = xr[i0] - u1r; t1i = xi[i0] - u1i;
          } else {
            t0r = xr[i0] + lamA * u1r; t0i = xi[i0] + lamA * u1i;
            t1r = xr[i0] - lamA * u1r; t1i = xi[i0] - lamA * u1i;
          }
          // t2, t3 = w x2 +- w^3 x3 = lamB (u2 +- rho u3), rho = lamC / lamB; then
          // y0, y2 = t0 +- t2 and y1, y3 = t1 +- (SIGN i) t3
          T u2r, u2i, u3r, u3i;
          const T lamB = tw_factor<SIGN>(mB, xr[i2], xi[i2], u2r, u2i);
          tw_factor<SIGN>(3 * mB, xr[i3], xi[i3], u3r, u3i);
          T pr, pi_, mr, mi;  // u2 + rho u3, u2 - rho u3
          if (mB % (kTw / 4) == 0) {  // then 3 mB is a quarter turn as well: no factors
            pr = u2r + u3r; pi_ = u2i + u3i;
            mr = u2r - u3r; mi = u2i - u3i;
          } else {
            const T rho = tw_rho<T>(mB);
            pr = u2r + rho * u3r; pi_ = u2i + rho * u3i;
            mr = u2r - rho * u3r; mi = u2i - rho * u3i;
          }
          T qr, qi;  // (SIGN i) (u2 - rho u3)
          qturn<T>(SIGN > 0 ? 1 : 3, mr, mi, qr, qi);
          if (mB % (kTw / 4) == 0) {
            xr[i0] = t0r + pr; xi[i0] = t0i + pi_;
            xr[i2] = t0r - pr; xi[i2] = t0i - pi_;
            xr[i1] = t1r + qr; xi[i1] = t1i + qi;
            xr[i3] = t1r - qr; xi[i3] = t1i - qi;
          } else {
            xr[i0] = t0r + lamB * pr; xi[i0] = t0i + lamB * pi_;
            xr[i2] = t0r - lamB * pr; xi[i2] = t0i - lamB * pi_;
            xr[i1] = t1r + lamB * qr; xi[i1] = t1i + lamB * qi;
            xr[i3] = t1r - lamB * qr; xi[i3] = t1i - lamB * qi;
          }
        }
      }
      fft_stages<N, SIGN, 4 * SPAN>(xr, xi);
    } else {
      constexpr int L = 2 * SPAN;
      constexpr int stride = kTw / L;
#pragma unroll
      for (int s = 0; s < N; s += L) {
#pragma unroll
        for (int k = 0; k < SPAN; ++k) {
          T tr, ti;
          twiddle<SIGN>(k * stride, xr[s + k + SPAN], xi[s + k + SPAN], tr, ti);
          xr[s + k + SPAN] = xr[s + k] - tr;
          xi[s + k + SPAN] = xi[s + k] - ti;
          xr[s + k] = xr[s + k] + tr;
          xi[s + k] = xi[s + k] + ti;
        }
      }
      fft_stages<N, SIGN, 2 * SPAN>(xr, xi);
    }
  }
}

// Power-of-two transform: bit reversal (register renaming), one radix-2 stage when
// log2 N is odd, then radix-4 stages.
template <int N, int SIGN, typename T>
__device__ __forceinline__ void fft_pow2(T (&xr)[N], T (&xi)[N]) {
  static_assert((N & (N - 1)) == 0 && N >= 1 && N <= 64, "power of two up to 64");
  if constexpr (N == 1) {
    return;
  } else {
    constexpr BitReverse<N> rev{};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int j = rev.v[i];
      if (j > i) {
        T t = xr[i]; xr[i] = xr[j]; xr[j] = t;
        t = xi[i]; xi[i] = xi[j]; xi[j] = t;
      }
    }
    constexpr bool odd = (N == 2) || (N == 8) || (N == 32);
    if constexpr (odd) {
#pragma unroll
      for (int s = 0; s < N; s += 2) {
        const T ar = xr[s], ai = xi[s];
        xr[s] = ar + xr[s + 1]; xi[s] = ai + xi[s + 1];
        xr[s + 1] = ar - xr[s + 1]; xi[s + 1] = ai - xi[s + 1];
      }
      fft_stages<N, SIGN, 2>(xr, xi);
    } else {
      fft_stages<N, SIGN, 1>(xr, xi);
    }
  }
}

// x_k <- sum_j x_j exp(SIGN 2 pi i j k / N); no scaling.  SIGN = -1 forward, +1 inverse.
// N = 3 P (P a power of two): a_r[m] = x[3m + r] are transformed with length P, then
// X[k + qP] = sum_r w3^{rq} W_N^{rk} A_r[k], w3 = exp(SIGN 2 pi i / 3).
template <int N, int SIGN, typename T>
__device__ __forceinline__ void fft_regs(T (&xr)[N], T (&xi)[N]) {
  if constexpr ((N & (N - 1)) == 0) {
    fft_pow2<N, SIGN>(xr, xi);
  } else {
    static_assert(N % 3 == 0 && ((N / 3) & (N / 3 - 1)) == 0 && N <= 48, "N = 3 * 2^k");
    constexpr int P = N / 3;
    T ar[3][P], ai[3][P];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int m = 0; m < P; ++m) {
        ar[r][m] = xr[3 * m + r];
        ai[r][m] = xi[3 * m + r];
      }
      fft_pow2<P, SIGN>(ar[r], ai[r]);
    }
    const T c3 = T(-0.5);  // cos(2 pi / 3)
    const T s3 = (SIGN > 0 ? T(1) : T(-1)) * tw_sin<T>(kTw / 3);  // SIGN sin(2 pi / 3)
    constexpr int stride = kTw / N;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      T b1r, b1i, b2r, b2i;
      twiddle<SIGN>(k * stride, ar[1][k], ai[1][k], b1r, b1i);
      twiddle<SIGN>(2 * k * stride, ar[2][k], ai[2][k], b2r, b2i);
      const T sr = b1r + b2r, si = b1i + b2i;  // b1 + b2
      const T dr = b1r - b2r, di = b1i - b2i;  // b1 - b2
      const T mr = ar[0][k] + c3 * sr, mi = ai[0][k] + c3 * si;
      // w3 b1 + w3^2 b2 = c3 (b1 + b2) + i s3 (b1 - b2), and its conjugate-rotation pair
      xr[k] = ar[0][k] + sr;
      xi[k] = ai[0][k] + si;
      xr[k + P] = mr - s3 * di;
      xi[k + P] = mi + s3 * dr;
      xr[k + 2 * P] = mr + s3 * di;
      xi[k + 2 * P] = mi - s3 * dr;
    }
  }
}

}  // namespace boltz

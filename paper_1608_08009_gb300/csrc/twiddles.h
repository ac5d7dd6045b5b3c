// Host-side twiddle tables of the register FFT (fft_regs.cuh): exp(2 pi i m / 192) and the
// factored form used by its radix-4 stages (Linzer and Feig, IBM J. Res. Dev. 37, 1993).
// Plain C++: the host table builder fills one copy and every kernel unit uploads it to
// its own constant memory.
#pragma once

#include <cmath>

namespace boltz {

constexpr int kTw = 192;  // lcm of every stage length the register transforms use

// Every twiddle table the register transforms read: cos, sin and the factored form
// (lam, mu, rho; see fft_regs.cuh), in float64 and rounded to float32.
struct TwiddleTables {
  double c64[kTw], s64[kTw], l64[kTw], m64[kTw], r64[kTw];
  float c32[kTw], s32[kTw], l32[kTw], m32[kTw], r32[kTw];
};

// Fills the host copy: theta = 2 pi m / 192 with the host libm in float64.
inline void fill_twiddle_tables(TwiddleTables& t) {
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < kTw; ++m) {
    const double th = 2.0 * pi * m / kTw;
    double c = std::cos(th), sn = std::sin(th);
    if (m % (kTw / 4) == 0) {  // exact quarter turns
      const int q = m / (kTw / 4);
      c = (q == 0) ? 1.0 : (q == 2) ? -1.0 : 0.0;
      sn = (q == 1) ? 1.0 : (q == 3) ? -1.0 : 0.0;
    }
    t.c64[m] = c;
    t.s64[m] = sn;
    const int r = m % (kTw / 2);
    const bool cos_form = (r <= kTw / 8) || (r >= 3 * kTw / 8);
    t.l64[m] = (m % (kTw / 4) == 0) ? 1.0 : cos_form ? c : sn;
    t.m64[m] = (m % (kTw / 4) == 0) ? 0.0 : cos_form ? sn / c : c / sn;
  }
  for (int m = 0; m < kTw; ++m) t.r64[m] = t.l64[(3 * m) % kTw] / t.l64[m];
  for (int m = 0; m < kTw; ++m) {
    t.c32[m] = (float)t.c64[m];
    t.s32[m] = (float)t.s64[m];
    t.l32[m] = (float)t.l64[m];
    t.m32[m] = (float)t.m64[m];
    t.r32[m] = (float)t.r64[m];
  }
}

}  // namespace boltz

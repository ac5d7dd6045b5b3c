// Host build of the kernels' register FFT (csrc/fft_regs.cuh compiled as plain C++), for
// the CPU test suite: every transform length the kernels use, both signs, in float64 and
// float32, against a direct float64 DFT; and the factored twiddle tables against
// exp(2 pi i m / 192).  Prints one JSON object.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <random>

#include "fft_regs.cuh"

using namespace boltz;

template <typename T, int N, int SIGN>
double rel_error(int trials) {
  std::mt19937 rng(1000 * N + 7 * SIGN + (int)sizeof(T));
  std::normal_distribution<double> d;
  double worst = 0;
  for (int t = 0; t < trials; ++t) {
    T xr[N], xi[N];
    std::complex<double> x[N];
    for (int i = 0; i < N; ++i) {
      xr[i] = (T)d(rng);
      xi[i] = (T)d(rng);
      x[i] = {(double)xr[i], (double)xi[i]};
    }
    fft_regs<N, SIGN>(xr, xi);
    double err = 0, nrm = 0;
    for (int k = 0; k < N; ++k) {
      std::complex<double> s = 0;
      for (int j = 0; j < N; ++j) {
        const double a = SIGN * 2.0 * M_PI * (double)((j * k) % N) / N;
        s += x[j] * std::complex<double>(std::cos(a), std::sin(a));
      }
      err = std::fmax(err, std::abs(s - std::complex<double>(xr[k], xi[k])));
      nrm = std::fmax(nrm, std::abs(s));
    }
    worst = std::fmax(worst, err / nrm);
  }
  return worst;
}

template <typename T, int N>
void report(const char* tag, int trials, bool* first) {
  printf("%s\"%s%d\": [%.3e, %.3e]", *first ? "" : ", ", tag, N, rel_error<T, N, -1>(trials),
         rel_error<T, N, +1>(trials));
  *first = false;
}

int main() {
  TwiddleTables t;
  fill_twiddle_tables(t);
  memcpy(c_twc64, t.c64, sizeof t.c64);
  memcpy(c_tws64, t.s64, sizeof t.s64);
  memcpy(c_twl64, t.l64, sizeof t.l64);
  memcpy(c_twm64, t.m64, sizeof t.m64);
  memcpy(c_twr64, t.r64, sizeof t.r64);
  memcpy(c_twc32, t.c32, sizeof t.c32);
  memcpy(c_tws32, t.s32, sizeof t.s32);
  memcpy(c_twl32, t.l32, sizeof t.l32);
  memcpy(c_twm32, t.m32, sizeof t.m32);
  memcpy(c_twr32, t.r32, sizeof t.r32);

  // factored form: exp(SIGN 2 pi i m / 192) x = lam u with u returned already turned
  double factor_err = 0;
  for (int sign = -1; sign <= 1; sign += 2)
    for (int m = 0; m < kTw; ++m) {
      const double a = sign * 2.0 * M_PI * m / kTw;
      const std::complex<double> w(std::cos(a), std::sin(a)), x(0.6, -0.8);
      double ur, ui, lam;
      if (sign > 0)
        lam = tw_factor<+1, double>(m, x.real(), x.imag(), ur, ui);
      else
        lam = tw_factor<-1, double>(m, x.real(), x.imag(), ur, ui);
      factor_err = std::fmax(factor_err, std::abs(lam * std::complex<double>(ur, ui) - w * x));
    }
  double rho_err = 0;
  for (int m = 0; m < kTw; ++m)
    if (m % (kTw / 4) != 0 && (3 * m) % (kTw / 4) != 0)
      rho_err = std::fmax(rho_err, std::fabs(t.r64[m] * t.l64[m] - t.l64[(3 * m) % kTw]));

  bool first = true;
  printf("{\"factor_err\": %.3e, \"rho_err\": %.3e, ", factor_err, rho_err);
  printf("\"f64\": {");
  report<double, 2>("N", 4, &first);
  report<double, 4>("N", 4, &first);
  report<double, 8>("N", 4, &first);
  report<double, 16>("N", 4, &first);
  report<double, 32>("N", 4, &first);
  report<double, 64>("N", 4, &first);
  report<double, 6>("N", 4, &first);
  report<double, 12>("N", 4, &first);
  report<double, 24>("N", 4, &first);
  report<double, 48>("N", 4, &first);
  printf("}, \"f32\": {");
  first = true;
  report<float, 8>("N", 50, &first);
  report<float, 16>("N", 50, &first);
  report<float, 32>("N", 50, &first);
  report<float, 64>("N", 50, &first);
  report<float, 24>("N", 50, &first);
  report<float, 48>("N", 50, &first);
  printf("}}\n");
  return 0;
}

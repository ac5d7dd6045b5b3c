// Host (float64) builder of the grid tables of the fast spectral collision operator.
//
// Paper: arxiv 1608.08009, Sec. 3.3 (truncation and periodisation rule, Fourier modes,
// Carleman representation Eq. FKM, decoupling Eq. decoup, 3D decoupling formula with the
// hard-sphere phi, half-sphere product quadrature) and Sec. 3.2 (projection, Eq. minim1).
//
// Readings taken where the paper is silent or inconsistent:
//  * S = 2L/(3 + sqrt 2) (the periodisation rule with T = L), Carleman radius R = 2S.
//  * psi(s) = 2 pi R J1(R s) / s, the Fourier transform of the disk of radius R in the
//    plane orthogonal to e (the printed psi puts the sin(theta) of the outer area
//    element inside the inner integral).
//  * direction sets on the half sphere: see boltz_grid_opts::dirs_kind.
//  * gamma != 1: Btilde = 4 C (|x|^2 + |y|^2)^((gamma-1)/2) is expanded over r
//    Gauss-Legendre nodes rho_r of |x| in [0, R]:
//      alpha_{j,r}(k)  = 2 u_r rho_r cos(rho_r xi_k . e_j)
//      alpha'_{j,r}(k) = 2 pi int_0^R rho' Btilde(rho_r, rho') J0(rho' |Pi xi_k|) d rho'.
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace boltz {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes (ascending) and weights on [a, b]: Newton iteration on the
// three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& u) {
  x.assign(n, 0.0);
  u.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0; p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    // node i of the descending sequence -> ascending index n-1-i
    x[n - 1 - i] = 0.5 * (b - a) * z + 0.5 * (b + a);
    u[n - 1 - i] = 0.5 * (b - a) * 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int product_a1(int M, int a1) {
  if (a1 > 0) return (M % a1 == 0) ? a1 : -1;
  for (int a = 1; a <= M; ++a)
    if (M % a == 0 && a * a >= M) return a;
  return -1;
}

double sinc(double x) {
  if (std::fabs(x) < 1e-8) return 1.0 - x * x / 6.0;
  return std::sin(x) / x;
}

// phi(s) = int_{-R}^{R} |rho| e^{i rho s} d rho = R^2 [2 Sinc(R s) - Sinc^2(R s / 2)]
double phi_hs(double s, double R) {
  double h = sinc(0.5 * R * s);
  return R * R * (2.0 * sinc(R * s) - h * h);
}

// psi(s) = 2 pi R J1(R s) / s
double psi_hs(double s, double R) {
  double x = R * s;
  double ratio = (std::fabs(x) < 1e-6) ? 0.5 - x * x / 16.0 : std::cyl_bessel_j(1.0, x) / x;
  return 2.0 * kPi * R * R * ratio;
}

// |Pi_{e-perp} xi| = |xi x e| for unit e; the cross product stays accurate when xi is
// nearly parallel to e, where sqrt(|xi|^2 - (xi . e)^2) cancels.
double perp_norm(double kx, double ky, double kz, double e0, double e1, double e2) {
  const double cx = ky * e2 - kz * e1;
  const double cy = kz * e0 - kx * e2;
  const double cz = kx * e1 - ky * e0;
  return std::sqrt(cx * cx + cy * cy + cz * cz);
}

int invert5(const double* A, double* G) {
  double m[5][10];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 10; ++j) m[i][j] = (j < 5) ? A[i * 5 + j] : (j - 5 == i ? 1.0 : 0.0);
  for (int c = 0; c < 5; ++c) {
    int p = c;
    for (int r = c + 1; r < 5; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[p][c])) p = r;
    if (m[p][c] == 0.0) return -1;
    if (p != c)
      for (int j = 0; j < 10; ++j) std::swap(m[p][j], m[c][j]);
    double d = m[c][c];
    for (int j = 0; j < 10; ++j) m[c][j] /= d;
    for (int r = 0; r < 5; ++r) {
      if (r == c) continue;
      double fct = m[r][c];
      if (fct != 0.0)
        for (int j = 0; j < 10; ++j) m[r][j] -= fct * m[c][j];
    }
  }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) G[i * 5 + j] = m[i][j + 5];
  return 0;
}

template <typename F>
void parallel_for(int n, F&& fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::max(1u, std::min(hw, 16u));
  if (nt > n) nt = n;
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int i = t; i < n; i += nt) fn(i);
    });
  for (auto& x : th) x.join();
}

}  // namespace

boltz_status build_tables(boltz_grid_s* g) {
  const int N = g->N, M = g->M;
  const size_t n = (size_t)N * N * N;
  g->dv = 2.0 * g->L / N;
  g->S = 2.0 * g->L / (3.0 + std::sqrt(2.0));
  if (!(g->R > 0)) g->R = 2.0 * g->S;
  const double R = g->R;

  // ---- direction set on the half sphere ------------------------------------------
  g->e.assign((size_t)M * 3, 0.0);
  g->wdir.assign(M, 0.0);
  if (g->dirs_kind == 0 || g->dirs_kind == 2) {
    int A1 = product_a1(M, g->a1);
    if (A1 <= 0) {
      set_error("dirs_a1 must divide M_dirs");
      return BOLTZ_EINVAL;
    }
    int A2 = M / A1;
    std::vector<double> ct, ut;
    if (g->dirs_kind == 2) gauss_legendre(A1, -1.0, 1.0, ct, ut);
    for (int p = 0; p < A1; ++p)
      for (int q = 0; q < A2; ++q) {
        int j = p * A2 + q;
        double vp = (q + 0.5) * kPi / A2;
        double st, c, w;
        if (g->dirs_kind == 0) {
          double th = (p + 0.5) * kPi / A1;
          st = std::sin(th);
          c = std::cos(th);
          w = (kPi / A1) * (kPi / A2) * st;
        } else {
          c = ct[p];
          st = std::sqrt(1.0 - c * c);
          w = ut[p] * (kPi / A2);
        }
        g->e[3 * j + 0] = st * std::cos(vp);
        g->e[3 * j + 1] = st * std::sin(vp);
        g->e[3 * j + 2] = c;
        g->wdir[j] = w;
      }
  } else if (g->dirs_kind == 1) {
    const double golden = kPi * (3.0 - std::sqrt(5.0));
    for (int j = 0; j < M; ++j) {
      double z = 1.0 - (j + 0.5) / M;
      double r = std::sqrt(1.0 - z * z);
      double ang = j * golden;
      g->e[3 * j + 0] = r * std::cos(ang);
      g->e[3 * j + 1] = r * std::sin(ang);
      g->e[3 * j + 2] = z;
      g->wdir[j] = 2.0 * kPi / M;
    }
  } else {
    set_error("dirs_kind must be 0, 1 or 2");
    return BOLTZ_EINVAL;
  }

  // ---- wave numbers ----------------------------------------------------------------
  std::vector<double> xi(N);
  for (int i = 0; i < N; ++i) xi[i] = kPi * (i < N / 2 ? i : i - N) / g->L;

  const int rank = g->rank;
  const int Meff = M * rank;
  g->M_eff = Meff;
  g->w.assign(Meff, 0.0);
  for (int j = 0; j < M; ++j)
    for (int r = 0; r < rank; ++r) g->w[(size_t)j * rank + r] = g->wdir[j];
  try {
    g->alpha.assign((size_t)Meff * n, 0.0);
    g->alphap.assign((size_t)Meff * n, 0.0);
    g->D.assign(n, 0.0);
  } catch (...) {
    set_error("host allocation of the kernel tables failed");
    return BOLTZ_ENOMEM;
  }

  if (rank == 1) {
    if (g->gamma != 1.0) {
      set_error("radial_rank 1 is exact only for gamma = 1");
      return BOLTZ_EINVAL;
    }
    const double bt = 4.0 * g->C_gamma;
    parallel_for(M, [&](int j) {
      const double e0 = g->e[3 * j], e1 = g->e[3 * j + 1], e2 = g->e[3 * j + 2];
      double* al = &g->alpha[(size_t)j * n];
      double* ap = &g->alphap[(size_t)j * n];
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b)
          for (int c = 0; c < N; ++c) {
            size_t idx = ((size_t)a * N + b) * N + c;
            double s = xi[a] * e0 + xi[b] * e1 + xi[c] * e2;
            double perp = perp_norm(xi[a], xi[b], xi[c], e0, e1, e2);
            al[idx] = bt * phi_hs(s, R);
            ap[idx] = psi_hs(perp, R);
          }
    });
  } else {
    std::vector<double> rho, u, rq, uq;
    gauss_legendre(rank, 0.0, R, rho, u);
    gauss_legendre(g->inner_nodes, 0.0, R, rq, uq);
    const int nq = g->inner_nodes;
    // gq[r][q] = u_q rho'_q Btilde(rho_r, rho'_q)
    std::vector<double> gq((size_t)rank * nq);
    for (int r = 0; r < rank; ++r)
      for (int q = 0; q < nq; ++q)
        gq[(size_t)r * nq + q] = uq[q] * rq[q] * 4.0 * g->C_gamma *
                                 std::pow(rho[r] * rho[r] + rq[q] * rq[q], 0.5 * (g->gamma - 1.0));
    parallel_for(M, [&](int j) {
      const double e0 = g->e[3 * j], e1 = g->e[3 * j + 1], e2 = g->e[3 * j + 2];
      std::vector<double> j0(nq);
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b)
          for (int c = 0; c < N; ++c) {
            size_t idx = ((size_t)a * N + b) * N + c;
            double s = xi[a] * e0 + xi[b] * e1 + xi[c] * e2;
            double perp = perp_norm(xi[a], xi[b], xi[c], e0, e1, e2);
            for (int q = 0; q < nq; ++q) j0[q] = std::cyl_bessel_j(0.0, rq[q] * perp);
            for (int r = 0; r < rank; ++r) {
              size_t i = (size_t)j * rank + r;
              g->alpha[i * n + idx] = 2.0 * u[r] * rho[r] * std::cos(rho[r] * s);
              double acc = 0.0;
              const double* gr = &gq[(size_t)r * nq];
              for (int q = 0; q < nq; ++q) acc += gr[q] * j0[q];
              g->alphap[i * n + idx] = 2.0 * kPi * acc;
            }
          }
    });
  }

  // D(k) = sum_i w_i alpha_i(k) alpha'_i(k): the Carleman loss multiplier K(k, k)
  for (int i = 0; i < Meff; ++i) {
    const double wi = g->w[i];
    const double* al = &g->alpha[(size_t)i * n];
    const double* ap = &g->alphap[(size_t)i * n];
    for (size_t k = 0; k < n; ++k) g->D[k] += wi * al[k] * ap[k];
  }

  // ---- projection matrix G = (Phi Phi^T)^-1 ----------------------------------------
  double A[25] = {0};
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b)
      for (int c = 0; c < N; ++c) {
        double vx = -g->L + a * g->dv, vy = -g->L + b * g->dv, vz = -g->L + c * g->dv;
        double phi[5] = {1.0, vx, vy, vz, 0.5 * (vx * vx + vy * vy + vz * vz)};
        for (int r = 0; r < 5; ++r)
          for (int s = 0; s < 5; ++s) A[r * 5 + s] += phi[r] * phi[s];
      }
  if (invert5(A, g->proj.G) != 0) {
    set_error("singular projection matrix");
    return BOLTZ_EINVAL;
  }
  return BOLTZ_OK;
}

// Two dimensions, Maxwell molecules (Sec. 3.3, dimension two; Eq. dfor0): Btilde is the
// constant 2 C_gamma (Eq. Btilde with d_v = 2, gamma = 0), angles theta_p = pi p / A with
// weight pi / A, alpha_p(k) = Btilde phi2(xi_k . e_p), alpha'_p(k) = phi2(xi_k . e_p-perp)
// with phi2(s) = int_{-R}^{R} e^{i rho s} d rho = 2 R Sinc(R s); D = sum_p w_p alpha_p
// alpha'_p.  Tables in (kx, ky) FFT storage order.  The projection uses the invariants
// (1, v_x, v_y, |v|^2/2); its 4x4 inverse sits in the 5x5 slots {0, 1, 2, 4} of G (row and
// column 3, the absent v_z, are zero).
boltz_status build_tables2d(boltz_grid_s* g) {
  const int N = g->N, M = g->M;
  const size_t n = (size_t)N * N;
  g->dv = 2.0 * g->L / N;
  g->S = 2.0 * g->L / (3.0 + std::sqrt(2.0));
  if (!(g->R > 0)) g->R = 2.0 * g->S;
  const double R = g->R;
  const double bt = 2.0 * g->C_gamma;
  g->rank = 1;
  g->M_eff = M;
  g->e.assign((size_t)M * 3, 0.0);
  g->wdir.assign(M, kPi / M);
  g->w.assign(M, kPi / M);
  try {
    g->alpha.assign((size_t)M * n, 0.0);
    g->alphap.assign((size_t)M * n, 0.0);
    g->D.assign(n, 0.0);
  } catch (...) {
    set_error("host allocation of the kernel tables failed");
    return BOLTZ_ENOMEM;
  }
  std::vector<double> xi(N);
  for (int i = 0; i < N; ++i) xi[i] = kPi * (i < N / 2 ? i : i - N) / g->L;
  for (int p = 0; p < M; ++p) {
    const double th = kPi * p / M, c = std::cos(th), sn = std::sin(th);
    g->e[3 * p + 0] = c;
    g->e[3 * p + 1] = sn;
    double* al = &g->alpha[(size_t)p * n];
    double* ap = &g->alphap[(size_t)p * n];
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b) {
        const size_t idx = (size_t)a * N + b;
        al[idx] = bt * 2.0 * R * sinc(R * (xi[a] * c + xi[b] * sn));
        ap[idx] = 2.0 * R * sinc(R * (-xi[a] * sn + xi[b] * c));
      }
  }
  for (int p = 0; p < M; ++p)
    for (size_t k = 0; k < n; ++k) g->D[k] += g->w[p] * g->alpha[(size_t)p * n + k] * g->alphap[(size_t)p * n + k];
  double A[25] = {0};
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double vx = -g->L + a * g->dv, vy = -g->L + b * g->dv;
      const double phi[5] = {1.0, vx, vy, 0.0, 0.5 * (vx * vx + vy * vy)};
      for (int r = 0; r < 5; ++r)
        for (int q = 0; q < 5; ++q) A[r * 5 + q] += phi[r] * phi[q];
    }
  A[3 * 5 + 3] = 1.0;  // placeholder for the absent v_z row; removed from G below
  if (invert5(A, g->proj.G) != 0) {
    set_error("singular projection matrix");
    return BOLTZ_EINVAL;
  }
  g->proj.G[3 * 5 + 3] = 0.0;
  return BOLTZ_OK;
}

}  // namespace boltz

// Host check of the hand-written reverse mode of the point fluxes
// (csrc/gks_point_adj.cuh) against forward-mode dual numbers run through the
// forward flux templates (csrc/gks_point.cuh): for random physical states and
// random output cotangents w, every component of the VJP J^T w must equal the
// directional derivative w . (J e_j); the F_t-only sweeps (FTO: a zero
// cotangent of F, the S2O4 adjoint's second stage) are given a random F
// cotangent, which they must ignore, and compared with w . (J e_j) for the
// F_t part of w alone.  Prints the largest relative error per case; exit
// status 1 if any exceeds 1e-11.
#define DG_HD inline
#include <cmath>
#include <cstdio>
#include <random>

struct Dl {
  double v, d;
  Dl() : v(0.0), d(0.0) {}
  Dl(double x) : v(x), d(0.0) {}
  Dl(double x, double dx) : v(x), d(dx) {}
};
inline Dl operator+(Dl a, Dl b) { return Dl(a.v + b.v, a.d + b.d); }
inline Dl operator-(Dl a, Dl b) { return Dl(a.v - b.v, a.d - b.d); }
inline Dl operator-(Dl a) { return Dl(-a.v, -a.d); }
inline Dl operator*(Dl a, Dl b) { return Dl(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dl operator/(Dl a, Dl b) {
  const double q = a.v / b.v;
  return Dl(q, (a.d - q * b.d) / b.v);
}
inline Dl& operator+=(Dl& a, Dl b) { return a = a + b; }
inline bool operator>(Dl a, Dl b) { return a.v > b.v; }
inline bool operator<(Dl a, Dl b) { return a.v < b.v; }
inline bool operator!=(Dl a, Dl b) { return a.v != b.v; }
inline Dl exp(Dl a) {
  const double e = std::exp(a.v);
  return Dl(e, e * a.d);
}
inline Dl sqrt(Dl a) {
  const double r = std::sqrt(a.v);
  return Dl(r, a.d / (2.0 * r));
}
inline Dl erfc(Dl a) { return Dl(std::erfc(a.v), -2.0 / std::sqrt(M_PI) * std::exp(-a.v * a.v) * a.d); }

#include "gks_point.cuh"
#include "gks_point_adj.cuh"

using namespace dghgks;

static std::mt19937_64 rng(2202);
static double uni(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

static void state(double q[5], double dq[3][5]) {
  const double rho = uni(0.7, 1.3), U = uni(-0.6, 0.6), V = uni(-0.6, 0.6), W = uni(-0.6, 0.6), p = uni(0.5, 1.5);
  q[0] = rho;
  q[1] = rho * U;
  q[2] = rho * V;
  q[3] = rho * W;
  q[4] = p / 0.4 + 0.5 * rho * (U * U + V * V + W * W);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k) dq[i][k] = uni(-0.3, 0.3) * (k == 4 ? 3.0 : 1.0);
}

template <class R>
static GasPar<R> gas(double mu, double pr, double dt, double tau_eps) {
  GasPar<R> g;
  g.K = 2.0;
  g.gm1 = 0.4;
  g.mu = mu;
  g.tau_add = tau_eps * dt;
  g.pr_fix = 1.0 / pr - 1.0;
  g.dt = dt;
  g.inv_dt = 1.0 / dt;
  return g;
}

template <bool FTO>
static double face_case(double mu, double pr, double dt, double tau_eps) {
  double qL[5], dqL[3][5], qR[5], dqR[3][5], Fb[5], Ftb[5];
  state(qL, dqL);
  state(qR, dqR);
  for (int k = 0; k < 5; ++k) {
    Fb[k] = uni(-1, 1);
    Ftb[k] = uni(-1, 1);
  }
  const GasPar<double> g = gas<double>(mu, pr, dt, tau_eps);
  double qLb[5], dqLb[3][5], qRb[5], dqRb[3][5], mub = 0.0;
  iface_flux_vjp<double, FTO>(qL, dqL, qR, dqR, g, Fb, Ftb, qLb, dqLb, qRb, dqRb, mub);
  double rev[41];
  for (int k = 0; k < 5; ++k) {
    rev[k] = qLb[k];
    rev[20 + k] = qRb[k];
    for (int i = 0; i < 3; ++i) {
      rev[5 + 5 * i + k] = dqLb[i][k];
      rev[25 + 5 * i + k] = dqRb[i][k];
    }
  }
  rev[40] = mub;
  double err = 0.0, scale = 0.0;
  for (int j = 0; j < 41; ++j) {
    Dl xL[5], dxL[3][5], xR[5], dxR[3][5], F[5], Ft[5];
    for (int k = 0; k < 5; ++k) {
      xL[k] = Dl(qL[k], j == k);
      xR[k] = Dl(qR[k], j == 20 + k);
      for (int i = 0; i < 3; ++i) {
        dxL[i][k] = Dl(dqL[i][k], j == 5 + 5 * i + k);
        dxR[i][k] = Dl(dqR[i][k], j == 25 + 5 * i + k);
      }
    }
    GasPar<Dl> gd = gas<Dl>(mu, pr, dt, tau_eps);
    gd.mu = Dl(mu, j == 40);
    iface_flux(xL, dxL, xR, dxR, gd, F, Ft);
    double fwd = 0.0;
    for (int k = 0; k < 5; ++k) fwd += (FTO ? 0.0 : Fb[k] * F[k].d) + Ftb[k] * Ft[k].d;
    err = std::fmax(err, std::fabs(fwd - rev[j]));
    scale = std::fmax(scale, std::fabs(fwd));
  }
  return err / scale;
}

template <bool FTO>
static double cell_case(double mu, double pr, double dt, double tau_eps) {
  double q[5], dq[3][5], Fb[3][5], Ftb[3][5];
  state(q, dq);
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 5; ++k) {
      Fb[d][k] = uni(-1, 1);
      Ftb[d][k] = uni(-1, 1);
    }
  const GasPar<double> g = gas<double>(mu, pr, dt, tau_eps);
  double qb[5], dqb[3][5], mub = 0.0;
  interior_flux_vjp<double, FTO>(q, dq, g, Fb, Ftb, qb, dqb, mub);
  double rev[21];
  for (int k = 0; k < 5; ++k) {
    rev[k] = qb[k];
    for (int i = 0; i < 3; ++i) rev[5 + 5 * i + k] = dqb[i][k];
  }
  rev[20] = mub;
  double err = 0.0, scale = 0.0;
  for (int j = 0; j < 21; ++j) {
    Dl x[5], dx[3][5], F[3][5], Ft[3][5];
    for (int k = 0; k < 5; ++k) {
      x[k] = Dl(q[k], j == k);
      for (int i = 0; i < 3; ++i) dx[i][k] = Dl(dq[i][k], j == 5 + 5 * i + k);
    }
    GasPar<Dl> gd = gas<Dl>(mu, pr, dt, tau_eps);
    gd.mu = Dl(mu, j == 20);
    interior_flux(x, dx, gd, F, Ft);
    double fwd = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < 5; ++k) fwd += (FTO ? 0.0 : Fb[d][k] * F[d][k].d) + Ftb[d][k] * Ft[d][k].d;
    err = std::fmax(err, std::fabs(fwd - rev[j]));
    scale = std::fmax(scale, std::fabs(fwd));
  }
  return err / scale;
}

int main() {
  const double cases[][4] = {{1e-2, 1.0, 1e-2, 0.0}, {1e-2, 0.72, 1e-2, 0.0}, {1e-3, 0.72, 5e-3, 0.05},
                             {0.0, 1.0, 1e-2, 0.01}, {5e-2, 0.72, 2e-3, 0.0}};
  double worst = 0.0;
  for (auto& c : cases)
    for (int rep = 0; rep < 4; ++rep) {
      const double ef = face_case<false>(c[0], c[1], c[2], c[3]);
      const double ec = cell_case<false>(c[0], c[1], c[2], c[3]);
      const double ef2 = face_case<true>(c[0], c[1], c[2], c[3]);
      const double ec2 = cell_case<true>(c[0], c[1], c[2], c[3]);
      std::printf("mu %g Pr %g dt %g tau_eps %g: face %.3e cell %.3e; F_t only: face %.3e cell %.3e\n", c[0], c[1],
                  c[2], c[3], ef, ec, ef2, ec2);
      worst = std::fmax(std::fmax(worst, std::fmax(ef, ec)), std::fmax(ef2, ec2));
    }
  std::printf("worst %.3e\n", worst);
  return worst <= 1e-11 ? 0 : 1;
}

// C entry points of the DG-HGKS oracle (TEST INFRASTRUCTURE ONLY; see
// dghgks_oracle.hpp).  Loaded by the tests, the smoke check and the CPU
// baseline leg of the benchmark through ctypes; never by the CUDA library.
//
// Return codes: 0 ok, -1 bad argument, -2 unsupported order / rule,
// -4 non-physical state (rho <= 0, p <= 0 or non-finite).
#include <cstdint>
#include <vector>

#include "dghgks_oracle.hpp"

using orc::Dual;

extern "C" {
typedef struct {
  int order, nq, nx, ny, nz;
  double lo[3], hi[3];
  double gamma, mu, Pr, tau_eps;
  // optional node coordinates per axis (n_d + 1 increasing values; NULL = uniform
  // cells between lo and hi); when given, lo/hi of that axis are taken from them
  const double* nodes[3];
} orc_cfg;
}

static bool make_grid(const orc_cfg* c, orc::Grid& G) {
  if (!c || c->order < 0 || c->order > 3 || c->nq < 1 || c->nq > 8 || c->nx < 1 || c->ny < 1 || c->nz < 1)
    return false;
  G.order = c->order;
  G.nq = c->nq;
  G.n[0] = c->nx;
  G.n[1] = c->ny;
  G.n[2] = c->nz;
  for (int d = 0; d < 3; ++d) {
    G.lo[d] = c->lo[d];
    G.hi[d] = c->hi[d];
    if (c->nodes[d]) {
      G.nodes[d].assign(c->nodes[d], c->nodes[d] + G.n[d] + 1);
      for (int q = 0; q < G.n[d]; ++q)
        if (!(G.nodes[d][q + 1] > G.nodes[d][q])) return false;
      G.lo[d] = G.nodes[d].front();
      G.hi[d] = G.nodes[d].back();
    }
    if (!(G.hi[d] > G.lo[d])) return false;
  }
  return true;
}

template <class T>
static orc::Phys<T> make_phys(const orc_cfg* c, T mu) {
  orc::Phys<T> p;
  p.gamma = c->gamma;
  p.K = (5.0 - 3.0 * c->gamma) / (c->gamma - 1.0);
  p.mu = mu;
  p.Pr = c->Pr;
  p.tau_eps = c->tau_eps;
  return p;
}

extern "C" {

int orc_n_modes(int order) { return orc::n_modes(order); }

int orc_gauss(int n, double* x, double* w) {
  if (n < 1 || n > 8) return -1;
  orc::gauss_rule(n, x, w);
  return 0;
}

// Basis values: out[m] = B_m(r), dout[m*3+d] = dB_m/dr_d at reference point r.
int orc_basis(int order, const double* r, double* out, double* dout) {
  auto md = orc::mode_list(order);
  for (size_t m = 0; m < md.size(); ++m) {
    out[m] = orc::basis(md[m], r);
    for (int d = 0; d < 3; ++d) dout[m * 3 + d] = orc::dbasis(md[m], r, d);
  }
  return 0;
}

// Moment tables of the Maxwellian (rho, U[3], lam): out = m[3][10] then xi[4].
int orc_moments(const double* U, double lam, int region, double K, double* out) {
  orc::Maxw<double> g;
  g.rho = 1.0;
  for (int d = 0; d < 3; ++d) g.U[d] = U[d];
  g.lam = lam;
  auto t = orc::moments(g, region, K);
  for (int d = 0; d < 3; ++d)
    for (int n = 0; n < orc::kMaxPow; ++n) out[d * orc::kMaxPow + n] = t.m[d][n];
  for (int j = 0; j < 4; ++j) out[3 * orc::kMaxPow + j] = t.xi[j];
  return 0;
}

// Slope a with <a psi> = b for the Maxwellian (U[3], lam) (normalised moments).
int orc_slope(const double* U, double lam, double K, const double* b, double* a) {
  orc::Maxw<double> g;
  g.rho = 1.0;
  for (int d = 0; d < 3; ++d) g.U[d] = U[d];
  g.lam = lam;
  auto t = orc::moments(g, 0, K);
  orc::slope_solve(t, b, a);
  return 0;
}

// Time-fit weights wF[6], wFt[6] of the six terms of Eq. (flux).
int orc_fit_weights(double tau, double dt, double* wF, double* wFt) {
  orc::fit_weights(tau, dt, wF, wFt);
  return 0;
}

// Interface flux across a face normal to axis dir (global frame); dQ are [3][5].
int orc_face_flux(int dir, const double* QL, const double* dQL, const double* QR, const double* dQR, double gamma,
                  double mu, double Pr, double tau_eps, double dt, double* F, double* Ft) {
  orc_cfg c{};
  c.gamma = gamma;
  c.mu = mu;
  c.Pr = Pr;
  c.tau_eps = tau_eps;
  auto ph = make_phys<double>(&c, mu);
  double dl[3][5], dr[3][5];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k) {
      dl[i][k] = dQL[i * 5 + k];
      dr[i][k] = dQR[i * 5 + k];
    }
  return orc::face_flux(dir, QL, dl, QR, dr, ph, dt, F, Ft) ? 0 : -4;
}

// Interior flux at a point: F, Ft are [3][5] (direction, variable).
int orc_cell_flux(const double* Q, const double* dQ, double gamma, double mu, double Pr, double tau_eps, double dt,
                  double* F, double* Ft) {
  orc_cfg c{};
  c.gamma = gamma;
  c.mu = mu;
  c.Pr = Pr;
  c.tau_eps = tau_eps;
  auto ph = make_phys<double>(&c, mu);
  double d[3][5], f[3][5], ft[3][5];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k) d[i][k] = dQ[i * 5 + k];
  if (!orc::cell_flux(Q, d, ph, dt, f, ft)) return -4;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k) {
      F[i * 5 + k] = f[i][k];
      Ft[i * 5 + k] = ft[i][k];
    }
  return 0;
}

int orc_residual(const orc_cfg* c, const double* Q, double dt, double* L, double* Lt) {
  orc::Grid G;
  if (!make_grid(c, G) || !(dt > 0)) return -1;
  auto ph = make_phys<double>(c, c->mu);
  return orc::residual(G, ph, Q, dt, L, Lt) ? 0 : -4;
}

// Residual of selected cells (flat cell index i + nx (j + ny k)); L, Lt are
// [ncells][5][n_modes].  A, At (may be NULL) receive the absolute-value scales.
int orc_residual_cells(const orc_cfg* c, const double* Q, double dt, const int64_t* cells, int64_t ncells, double* L,
                       double* Lt, double* A, double* At) {
  orc::Grid G;
  if (!make_grid(c, G) || !(dt > 0)) return -1;
  auto ph = make_phys<double>(c, c->mu);
  const int nm = G.nm();
  int rc = 0;
#pragma omp parallel for schedule(dynamic)
  for (int64_t s = 0; s < ncells; ++s) {
    int64_t id = cells[s];
    int i = (int)(id % G.n[0]), j = (int)((id / G.n[0]) % G.n[1]), k = (int)(id / ((int64_t)G.n[0] * G.n[1]));
    if (!orc::residual_cell(G, ph, Q, dt, i, j, k, L + s * 5 * nm, Lt + s * 5 * nm, A ? A + s * 5 * nm : nullptr,
                            At ? At + s * 5 * nm : nullptr)) {
#pragma omp atomic write
      rc = -4;
    }
  }
  return rc;
}

int orc_step(const orc_cfg* c, double* Q, double dt, int nsteps) {
  orc::Grid G;
  if (!make_grid(c, G) || !(dt > 0)) return -1;
  auto ph = make_phys<double>(c, c->mu);
  for (int s = 0; s < nsteps; ++s)
    if (!orc::s2o4_step(G, ph, Q, dt)) return -4;
  return 0;
}

int orc_totals(const orc_cfg* c, const double* Q, double* out) {
  orc::Grid G;
  if (!make_grid(c, G)) return -1;
  orc::totals(G, Q, out);
  return 0;
}

int orc_kinetic_energy(const orc_cfg* c, const double* Q, double rho0, double* Ek) {
  orc::Grid G;
  if (!make_grid(c, G)) return -1;
  *Ek = orc::kinetic_energy(G, Q, rho0);
  return 0;
}

int orc_enstrophy_dissipation(const orc_cfg* c, const double* Q, double rho0, double* eps) {
  orc::Grid G;
  if (!make_grid(c, G)) return -1;
  *eps = orc::enstrophy_dissipation(G, Q, c->mu, rho0);
  return 0;
}

int orc_project(const orc_cfg* c, int ic, const double* par, double* Q) {
  orc::Grid G;
  if (!make_grid(c, G) || ic < 1 || ic > 4) return -1;
  orc::project_ic(G, ic, par, c->gamma, Q);
  return 0;
}

int orc_density_errors(const orc_cfg* c, const double* Q, int ic, const double* par, double* out) {
  orc::Grid G;
  if (!make_grid(c, G) || ic < 1 || ic > 4) return -1;
  orc::density_errors(G, Q, ic, par, c->gamma, out);
  return 0;
}

// One S2O4 step of the scalar ODE dq/dt = lam q (L = lam q, L_t = lam^2 q),
// through the same stage combinations the grid step uses.
int orc_s2o4_scalar(double lam, double q0, double dt, double* out) {
  double L = lam * q0, Lt = lam * lam * q0;
  double qs = orc::s2o4_intermediate(q0, L, Lt, dt);
  double Lts = lam * lam * qs;
  *out = orc::s2o4_final(q0, L, Lt, Lts, dt);
  return 0;
}

// ---- forward-mode (dual number) derivatives, for the adjoint checks ----

// JVP of (L, L_t) at Q along (dQ, dmu).
int orc_residual_jvp(const orc_cfg* c, const double* Q, const double* dQ, double dmu, double dt, double* L, double* Lt,
                     double* dL, double* dLt) {
  orc::Grid G;
  if (!make_grid(c, G) || !(dt > 0)) return -1;
  const int64_t N = 5 * (int64_t)G.nm() * G.cells();
  std::vector<Dual<double>> q(N), l(N), lt(N);
  for (int64_t x = 0; x < N; ++x) q[x] = Dual<double>(Q[x], dQ[x]);
  auto ph = make_phys<Dual<double>>(c, Dual<double>(c->mu, dmu));
  if (!orc::residual(G, ph, q.data(), dt, l.data(), lt.data())) return -4;
  for (int64_t x = 0; x < N; ++x) {
    L[x] = l[x].v;
    dL[x] = l[x].d;
    Lt[x] = lt[x].v;
    dLt[x] = lt[x].d;
  }
  return 0;
}

// nsteps S2O4 steps of (Q, dQ) in place along the viscosity direction dmu;
// on return *Ek and *dEk hold E_k of the final state and its derivative.
int orc_step_jvp(const orc_cfg* c, double* Q, double* dQ, double dmu, double dt, int nsteps, double rho0, double* Ek,
                 double* dEk) {
  orc::Grid G;
  if (!make_grid(c, G) || !(dt > 0)) return -1;
  const int64_t N = 5 * (int64_t)G.nm() * G.cells();
  std::vector<Dual<double>> q(N);
  for (int64_t x = 0; x < N; ++x) q[x] = Dual<double>(Q[x], dQ[x]);
  auto ph = make_phys<Dual<double>>(c, Dual<double>(c->mu, dmu));
  for (int s = 0; s < nsteps; ++s)
    if (!orc::s2o4_step(G, ph, q.data(), dt)) return -4;
  for (int64_t x = 0; x < N; ++x) {
    Q[x] = q[x].v;
    dQ[x] = q[x].d;
  }
  Dual<double> e = orc::kinetic_energy(G, q.data(), rho0);
  *Ek = e.v;
  *dEk = e.d;
  return 0;
}

}  // extern "C"

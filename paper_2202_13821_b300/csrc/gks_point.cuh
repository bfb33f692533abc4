// Gas-kinetic flux at one quadrature point (device code, FP64 or FP32).
//
// Sec. 2 of arXiv:2202.13821: BGK model, Maxwellian g, psi = (1,u,v,w,
// (u^2+v^2+w^2+xi^2)/2), K = (5 - 3 gamma)/(gamma - 1) internal DOF.
//   * iface_flux: the interface distribution of Eq. (flux) with its slopes
//     a^k_i, A^k (k = l, r), the equilibrium Q_0 from the half-space moments
//     and its slopes abar_i, Abar; time-integrated over [0, dt] and
//     [0, dt/2] and fitted linearly in time (Eq. expansion-1) -> F, F_t.
//   * interior_flux: the simplified interior distribution of Eq. (flux-2),
//     f = g0 (1 - tau (a.u + A) + A t), which is linear in t: F = F(0),
//     F_t = rho <u_d A psi>.
//   * tau = mu / p + tau_eps dt (Sec. 3, Remark 1).
//   * Pr != 1 (not in the paper): the energy flux gains (1/Pr - 1) q, where
//     q = 1/2 <(u_n - U_n)(|u - U|^2 + xi^2) f> is evaluated from the flux
//     moments F = <u_n psi phi> and density moments W = <psi phi> of each
//     term phi of f.
//
// Implementation choices (B300): moment indices are template parameters so
// every moment product is resolved at compile time; the 5x5 slope systems are
// solved in closed form; side-local data is folded into running sums
// (Q_0, dQ_0/dn, and the free-transport flux moments) before the other side
// is touched, so the live register set stays small.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

// Point functions compile for the device and, for the operation counter, for
// the host with a counting scalar type.
#ifndef DG_HD
#define DG_HD __host__ __device__ __forceinline__
#endif

namespace dghgks {

using std::erfc;
using std::exp;
using std::sqrt;

// Division, reciprocal square root and exponential.  The FP64 path uses the
// IEEE operations; the FP32 path uses the single-instruction approximations
// of the special-function unit (about 2 ulp), which is well inside the
// FP32-mixed error budget and avoids the multi-instruction IEEE sequences.
template <class R>
DG_HD R fdiv(R a, R b) {
  return a / b;
}
template <class R>
DG_HD R frsqrt(R x) {
  return R(1) / sqrt(x);
}
template <class R>
DG_HD R fexp(R x) {
  return exp(x);
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) {
  return __fdividef(a, b);
}
template <>
__device__ __forceinline__ float frsqrt<float>(float x) {
  return rsqrtf(x);
}
template <>
__device__ __forceinline__ float fexp<float>(float x) {
  return __expf(x);
}
#endif

template <class R>
struct GasPar {
  R K;         // internal degrees of freedom
  R gm1;       // gamma - 1
  R mu;        // dynamic viscosity
  R tau_add;   // tau_eps * dt
  R pr_fix;    // 1/Pr - 1
  R dt;        // time step of the flux fit
  R inv_dt;
};

// Moment table of one Maxwellian: <u^n>, <v^n>, <w^n> (n <= 6), <xi^2>, <xi^4>,
// normalised by the density.
template <class R>
struct MomTab {
  R u[7], v[7], w[7];
  R xi2, xi4;
};

template <class R>
DG_HD void raw_moments_tail(R* m, R U, R h) {
  // <c^(n+2)> = U <c^(n+1)> + (n+1) h <c^n> with h = 1/(2 lambda)
#pragma unroll
  for (int n = 0; n < 5; ++n) m[n + 2] = U * m[n + 1] + R(n + 1) * h * m[n];
}

template <class R>
DG_HD void full_line(R* m, R U, R h) {
  m[0] = R(1);
  m[1] = U;
  raw_moments_tail(m, U, h);
}

// u > 0 (sgn = +1) or u < 0 (sgn = -1) half line
template <class R>
DG_HD void half_line(R* m, R U, R lam, R h, int sgn) {
  const R rs = frsqrt(lam);
  const R sl = lam * rs;  // sqrt(lam)
  const R e = fexp(-lam * U * U) * (R(0.28209479177387814347) * rs);  // exp(-lam U^2) / (2 sqrt(pi lam))
  const R sg = sgn > 0 ? R(1) : R(-1);  // u > 0 (sgn = +1) or u < 0 half space
  m[0] = R(0.5) * erfc(-sg * sl * U);
  m[1] = U * m[0] + sg * e;
  raw_moments_tail(m, U, h);
}

template <class R>
struct Prim {
  R rho, U, V, W, lam;
};

// conservative -> (rho, U, V, W, lambda = rho / 2p); false if rho or p is not positive
template <class R>
DG_HD bool prim_of(const R q[5], R gm1, Prim<R>& p) {
  const R ir = fdiv(R(1), q[0]);
  p.rho = q[0];
  p.U = q[1] * ir;
  p.V = q[2] * ir;
  p.W = q[3] * ir;
  const R pres = gm1 * (q[4] - R(0.5) * (q[1] * p.U + q[2] * p.V + q[3] * p.W));
  p.lam = fdiv(R(0.5) * q[0], pres);
  return (q[0] > R(0)) && (pres > R(0)) && (p.lam < R(1e30)) && (q[0] < R(1e30));
}

// ---- moments of products (compile-time powers) ----
template <int A, int B, int C, class R>
DG_HD R Gm(const MomTab<R>& t) {
  static_assert(A <= 6 && B <= 6 && C <= 6, "moment power out of table");
  return t.u[A] * t.v[B] * t.w[C];
}
// <u^A v^B w^C psi_5>
template <int A, int B, int C, class R>
DG_HD R G5(const MomTab<R>& t) {
  return R(0.5) * (Gm<A + 2, B, C>(t) + Gm<A, B + 2, C>(t) + Gm<A, B, C + 2>(t) + t.xi2 * Gm<A, B, C>(t));
}
// <u^A v^B w^C psi_5^2>
template <int A, int B, int C, class R>
DG_HD R G55(const MomTab<R>& t) {
  return R(0.25) * (Gm<A + 4, B, C>(t) + Gm<A, B + 4, C>(t) + Gm<A, B, C + 4>(t) +
                    R(2) * (Gm<A + 2, B + 2, C>(t) + Gm<A + 2, B, C + 2>(t) + Gm<A, B + 2, C + 2>(t)) +
                    R(2) * t.xi2 * (Gm<A + 2, B, C>(t) + Gm<A, B + 2, C>(t) + Gm<A, B, C + 2>(t)) +
                    t.xi4 * Gm<A, B, C>(t));
}

// out += s * <u^A v^B w^C psi>
template <int A, int B, int C, class R>
DG_HD void mom_psi(const MomTab<R>& t, R s, R out[5]) {
  out[0] += s * Gm<A, B, C>(t);
  out[1] += s * Gm<A + 1, B, C>(t);
  out[2] += s * Gm<A, B + 1, C>(t);
  out[3] += s * Gm<A, B, C + 1>(t);
  out[4] += s * G5<A, B, C>(t);
}

// out += s * <u^A v^B w^C (a . psi) psi>
template <int A, int B, int C, class R>
DG_HD void mom_a_psi(const MomTab<R>& t, const R a[5], R s, R out[5]) {
  out[0] += s * (a[0] * Gm<A, B, C>(t) + a[1] * Gm<A + 1, B, C>(t) + a[2] * Gm<A, B + 1, C>(t) +
                 a[3] * Gm<A, B, C + 1>(t) + a[4] * G5<A, B, C>(t));
  out[1] += s * (a[0] * Gm<A + 1, B, C>(t) + a[1] * Gm<A + 2, B, C>(t) + a[2] * Gm<A + 1, B + 1, C>(t) +
                 a[3] * Gm<A + 1, B, C + 1>(t) + a[4] * G5<A + 1, B, C>(t));
  out[2] += s * (a[0] * Gm<A, B + 1, C>(t) + a[1] * Gm<A + 1, B + 1, C>(t) + a[2] * Gm<A, B + 2, C>(t) +
                 a[3] * Gm<A, B + 1, C + 1>(t) + a[4] * G5<A, B + 1, C>(t));
  out[3] += s * (a[0] * Gm<A, B, C + 1>(t) + a[1] * Gm<A + 1, B, C + 1>(t) + a[2] * Gm<A, B + 1, C + 1>(t) +
                 a[3] * Gm<A, B, C + 2>(t) + a[4] * G5<A, B, C + 1>(t));
  out[4] += s * (a[0] * G5<A, B, C>(t) + a[1] * G5<A + 1, B, C>(t) + a[2] * G5<A, B + 1, C>(t) +
                 a[3] * G5<A, B, C + 1>(t) + a[4] * G55<A, B, C>(t));
}

// out += s * <u_D^(E) (a_x u + a_y v + a_z w) psi> with u_D^E = u^E (D=0), v^E (D=1), w^E (D=2)
template <int D, int E, class R>
DG_HD void mom_adotu_psi(const MomTab<R>& t, const R a[3][5], R s, R out[5]) {
  constexpr int A = (D == 0) ? E : 0, B = (D == 1) ? E : 0, C = (D == 2) ? E : 0;
  mom_a_psi<A + 1, B, C>(t, a[0], s, out);
  mom_a_psi<A, B + 1, C>(t, a[1], s, out);
  mom_a_psi<A, B, C + 1>(t, a[2], s, out);
}

template <int D, class R>
DG_HD void mom_ud_psi(const MomTab<R>& t, R s, R out[5]) {
  mom_psi<(D == 0), (D == 1), (D == 2)>(t, s, out);
}
template <int D, class R>
DG_HD void mom_ud_a_psi(const MomTab<R>& t, const R a[5], R s, R out[5]) {
  mom_a_psi<(D == 0), (D == 1), (D == 2)>(t, a, s, out);
}

template <class R>
DG_HD void full_table(const Prim<R>& p, R K, MomTab<R>& t) {
  const R h = fdiv(R(0.5), p.lam);
  full_line(t.u, p.U, h);
  full_line(t.v, p.V, h);
  full_line(t.w, p.W, h);
  t.xi2 = K * h;
  t.xi4 = K * (K + R(2)) * h * h;
}

// Closed-form solution of <a psi> = b for the Maxwellian p (normalised moments):
// with E = |U|^2 + (K+3)/(2 lam), r_i = b_{i} - U_i b_0 (i = 1..3),
// a_4 = 4 lam^2/(K+3) (2 b_4 - E b_0 - 2 U.r), a_i = 2 lam r_i - U_i a_4,
// a_0 = b_0 - U.a_{1..3} - a_4 E / 2.
template <class R>
DG_HD void slope_solve(const Prim<R>& p, R K, const R b[5], R a[5]) {
  const R E = p.U * p.U + p.V * p.V + p.W * p.W + fdiv((K + R(3)) * R(0.5), p.lam);
  const R r1 = b[1] - p.U * b[0], r2 = b[2] - p.V * b[0], r3 = b[3] - p.W * b[0];
  a[4] = fdiv(R(4) * p.lam * p.lam, K + R(3)) * (R(2) * b[4] - E * b[0] - R(2) * (p.U * r1 + p.V * r2 + p.W * r3));
  const R tl = R(2) * p.lam;
  a[1] = tl * r1 - p.U * a[4];
  a[2] = tl * r2 - p.V * a[4];
  a[3] = tl * r3 - p.W * a[4];
  a[0] = b[0] - p.U * a[1] - p.V * a[2] - p.W * a[3] - R(0.5) * a[4] * E;
}

// heat-flux moment of one term phi: 1/2 <(u_n - U_n)(|u-U|^2 + xi^2) phi> from
// F = <u_n psi phi>, W = <psi phi>; (U_n, Ut1, Ut2) = velocity, normal first.
template <class R>
DG_HD R heat_of(const R F[5], const R W[5], R Un, R Ut1, R Ut2, int n) {
  // components of psi: 1 -> U_n is component 1+n in the frame where F was taken
  const R U2 = Un * Un + Ut1 * Ut1 + Ut2 * Ut2;
  (void)n;
  return F[4] - Un * W[4] - (Un * F[1] + Ut1 * F[2] + Ut2 * F[3]) + Un * (Un * W[1] + Ut1 * W[2] + Ut2 * W[3]) +
         R(0.5) * U2 * (F[0] - Un * W[0]);
}

// Linear-in-time fit weights of the six terms of Eq. (flux): F = sum wF_j V_j,
// F_t = sum wFt_j V_j with V_j = (g0, (abar.u) g0, Abar g0, g_k, (a^k.u) g_k, A^k g_k)
// moments.  With Eh = exp(-dt/(2 tau)), s = 1 - Eh, x = tau/dt,
// phi = x s (2 + s) and q = 4 x s^2 / dt:
//   wF  = (1 - phi, 2 tau phi - tau (2 - s^2), tau phi - tau, phi, -2 tau phi + tau (1 - s^2), -tau phi)
//   wFt = (q, -2 tau q + 4 x Eh s, 1 - tau q, -q, 2 tau q - 4 x Eh s, tau q)
template <class R>
DG_HD void fit_weights(R tau, R dt, R inv_dt, R wF[6], R wFt[6]) {
  R Eh = R(0), x = R(0);
  if (tau > R(0)) {
    Eh = fexp(fdiv(R(-0.5) * dt, tau));
    x = tau * inv_dt;
  }
  const R s = R(1) - Eh;
  const R phi = x * s * (R(2) + s);
  const R q = R(4) * x * s * s * inv_dt;
  const R es = R(4) * x * Eh * s;
  wF[0] = R(1) - phi;
  wF[1] = R(2) * tau * phi - tau * (R(2) - s * s);
  wF[2] = tau * phi - tau;
  wF[3] = phi;
  wF[4] = -R(2) * tau * phi + tau * (R(1) - s * s);
  wF[5] = -tau * phi;
  wFt[0] = q;
  wFt[1] = -R(2) * tau * q + es;
  wFt[2] = R(1) - tau * q;
  wFt[3] = -q;
  wFt[4] = R(2) * tau * q - es;
  wFt[5] = tau * q;
}

// ---------------------------------------------------------------------------
// Interface flux (local frame: component 1 = normal).  q*, dq* are the traces
// and derivatives (n_1 = normal, n_2, n_3) of the left (u>0 upwind) and right
// states.  Returns false if a state is not physical.
// ---------------------------------------------------------------------------
template <class R>
struct SideSums {
  R Q0[5], dQ0[3][5];  // sum_k rho_k <psi>_k, sum_k rho_k <a^k_i psi>_k
  R V4[5], V5[5], V6[5];  // free-transport moments
  R W5[5], W6[5];         // density moments of terms 5 and 6 (Prandtl fix only)
};

// One side of the interface: SGN = +1 for the left state (its u > 0
// half-space reaches the interface), -1 for the right state.  SGN is a runtime
// value so that a kernel can loop over the two sides without unrolling.
template <class R>
DG_HD bool iface_side(int SGN, const R q[5], const R dq[3][5], const GasPar<R>& g, bool pr_fix,
                      SideSums<R>& S) {
  Prim<R> p;
  const bool ok = prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  R a[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R b[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k] = dq[i][k] * ir;
    slope_solve(p, g.K, b, a[i]);
  }
  MomTab<R> t;
  full_table(p, g.K, t);
  // compatibility: <A psi> = -<(a.u) psi>
  R bA[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_adotu_psi<0, 0>(t, a, R(-1), bA);
  R A[5];
  slope_solve(p, g.K, bA, A);
  // half-space table along the normal
  half_line(t.u, p.U, p.lam, fdiv(R(0.5), p.lam), SGN);
  const R r = p.rho;
  mom_psi<0, 0, 0>(t, r, S.Q0);
#pragma unroll
  for (int i = 0; i < 3; ++i) mom_a_psi<0, 0, 0>(t, a[i], r, S.dQ0[i]);
  mom_psi<1, 0, 0>(t, r, S.V4);
  mom_adotu_psi<0, 1>(t, a, r, S.V5);
  mom_a_psi<1, 0, 0>(t, A, r, S.V6);
  if (pr_fix) {
    mom_adotu_psi<0, 0>(t, a, r, S.W5);
    mom_a_psi<0, 0, 0>(t, A, r, S.W6);
  }
  return ok;
}

template <class R, int SGN>
DG_HD bool iface_side(const R q[5], const R dq[3][5], const GasPar<R>& g, bool pr_fix, SideSums<R>& S) {
  return iface_side<R>(SGN, q, dq, g, pr_fix, S);
}

template <class R>
DG_HD void iface_zero(SideSums<R>& S) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    S.Q0[k] = S.V4[k] = S.V5[k] = S.V6[k] = S.W5[k] = S.W6[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) S.dQ0[i][k] = R(0);
  }
}

// Equilibrium state g_0 of the interface, its slopes, tau, the time fit, and
// the flux (local frame) from the side sums of both sides.
template <class R>
DG_HD bool iface_finish(const SideSums<R>& S, const GasPar<R>& g, R F[5], R Ft[5]) {
  const bool pr_fix = (g.pr_fix != R(0));
  Prim<R> p0;
  const bool ok = prim_of(S.Q0, g.gm1, p0);
  const R ir0 = fdiv(R(1), p0.rho);
  R ab[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R b[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k] = S.dQ0[i][k] * ir0;
    slope_solve(p0, g.K, b, ab[i]);
  }
  MomTab<R> t0;
  full_table(p0, g.K, t0);
  R Wab[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_adotu_psi<0, 0>(t0, ab, R(1), Wab);  // <(abar.u) psi>
  R bA[5], Ab[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) bA[k] = -Wab[k];
  slope_solve(p0, g.K, bA, Ab);

  // collision time and fit weights
  const R tau = fdiv(g.mu * R(2) * p0.lam, p0.rho) + g.tau_add;  // mu / p_0 + tau_eps dt
  R wF[6], wFt[6];
  fit_weights(tau, g.dt, g.inv_dt, wF, wFt);

  R V1[5] = {R(0), R(0), R(0), R(0), R(0)}, V2[5] = {R(0), R(0), R(0), R(0), R(0)},
    V3[5] = {R(0), R(0), R(0), R(0), R(0)};
  const R r0 = p0.rho;
  mom_psi<1, 0, 0>(t0, r0, V1);
  mom_adotu_psi<0, 1>(t0, ab, r0, V2);
  mom_a_psi<1, 0, 0>(t0, Ab, r0, V3);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    F[k] = wF[0] * V1[k] + wF[1] * V2[k] + wF[2] * V3[k] + wF[3] * S.V4[k] + wF[4] * S.V5[k] + wF[5] * S.V6[k];
    Ft[k] = wFt[0] * V1[k] + wFt[1] * V2[k] + wFt[2] * V3[k] + wFt[3] * S.V4[k] + wFt[4] * S.V5[k] +
            wFt[5] * S.V6[k];
  }
  if (pr_fix) {
    // heat moments of terms 2..6 about U_0 (term 1, g_0 itself, carries none)
    R W2[5], W3[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      W2[k] = r0 * Wab[k];
      W3[k] = -r0 * Wab[k];
    }
    const R H2 = heat_of(V2, W2, p0.U, p0.V, p0.W, 0);
    const R H3 = heat_of(V3, W3, p0.U, p0.V, p0.W, 0);
    const R H4 = heat_of(S.V4, S.Q0, p0.U, p0.V, p0.W, 0);
    const R H5 = heat_of(S.V5, S.W5, p0.U, p0.V, p0.W, 0);
    const R H6 = heat_of(S.V6, S.W6, p0.U, p0.V, p0.W, 0);
    F[4] += g.pr_fix * (wF[1] * H2 + wF[2] * H3 + wF[3] * H4 + wF[4] * H5 + wF[5] * H6);
    Ft[4] += g.pr_fix * (wFt[1] * H2 + wFt[2] * H3 + wFt[3] * H4 + wFt[4] * H5 + wFt[5] * H6);
  }
  return ok;
}

template <class R>
DG_HD bool iface_flux(const R qL[5], const R dqL[3][5], const R qR[5], const R dqR[3][5], const GasPar<R>& g, R F[5],
                      R Ft[5]) {
  const bool pr_fix = (g.pr_fix != R(0));
  SideSums<R> S;
  iface_zero(S);
  bool ok = iface_side<R, +1>(qL, dqL, g, pr_fix, S);
  ok = iface_side<R, -1>(qR, dqR, g, pr_fix, S) && ok;
  return iface_finish(S, g, F, Ft) && ok;
}

// ---------------------------------------------------------------------------
// Interior flux of Eq. (flux-2) in the global frame: F[d][k], Ft[d][k].
// ---------------------------------------------------------------------------
template <int D, class R>
DG_HD void interior_dir(const MomTab<R>& t, const Prim<R>& p, const R a[3][5], const R A[5],
                                             const R Wau[5], R tau, const GasPar<R>& g, R F[5], R Ft[5]) {
  R m0[5] = {R(0), R(0), R(0), R(0), R(0)}, m1[5] = {R(0), R(0), R(0), R(0), R(0)},
    m2[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_ud_psi<D>(t, R(1), m0);
  mom_adotu_psi<D, 1>(t, a, R(1), m1);
  mom_ud_a_psi<D>(t, A, R(1), m2);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    F[k] = p.rho * (m0[k] - tau * (m1[k] + m2[k]));
    Ft[k] = p.rho * m2[k];
  }
  if (g.pr_fix != R(0)) {
    // velocity ordered with the flux direction first
    const R Un = (D == 0) ? p.U : (D == 1) ? p.V : p.W;
    R Fm1[5], Fm2[5], Wm2[5];
    // heat_of expects momentum flux components in global order with U_n first; build
    // the frame-aligned copies: (psi_0, u_n, u_t1, u_t2, psi_5) with t1, t2 = the other axes
    constexpr int e1 = (D == 0) ? 2 : 1, e2 = (D == 2) ? 2 : 3;
    constexpr int en = 1 + D;
    Fm1[0] = m1[0];
    Fm1[1] = m1[en];
    Fm1[2] = m1[e1];
    Fm1[3] = m1[e2];
    Fm1[4] = m1[4];
    Fm2[0] = m2[0];
    Fm2[1] = m2[en];
    Fm2[2] = m2[e1];
    Fm2[3] = m2[e2];
    Fm2[4] = m2[4];
    R Wm1[5];
    Wm1[0] = Wau[0];
    Wm1[1] = Wau[en];
    Wm1[2] = Wau[e1];
    Wm1[3] = Wau[e2];
    Wm1[4] = Wau[4];
#pragma unroll
    for (int k = 0; k < 5; ++k) Wm2[k] = -Wm1[k];
    const R Ut1 = (e1 == 1) ? p.U : (e1 == 2) ? p.V : p.W;
    const R Ut2 = (e2 == 1) ? p.U : (e2 == 2) ? p.V : p.W;
    const R H1 = heat_of(Fm1, Wm1, Un, Ut1, Ut2, 0);
    const R H2 = heat_of(Fm2, Wm2, Un, Ut1, Ut2, 0);
    F[4] += g.pr_fix * p.rho * (-tau * (H1 + H2));
    Ft[4] += g.pr_fix * p.rho * H2;
  }
}

template <class R>
DG_HD bool interior_flux(const R q[5], const R dq[3][5], const GasPar<R>& g, R F[3][5],
                                              R Ft[3][5]) {
  Prim<R> p;
  const bool ok = prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  R a[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R b[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k] = dq[i][k] * ir;
    slope_solve(p, g.K, b, a[i]);
  }
  MomTab<R> t;
  full_table(p, g.K, t);
  R Wau[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_adotu_psi<0, 0>(t, a, R(1), Wau);
  R bA[5], A[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) bA[k] = -Wau[k];
  slope_solve(p, g.K, bA, A);
  const R tau = fdiv(g.mu * R(2) * p.lam, p.rho) + g.tau_add;
  interior_dir<0>(t, p, a, A, Wau, tau, g, F[0], Ft[0]);
  interior_dir<1>(t, p, a, A, Wau, tau, g, F[1], Ft[1]);
  interior_dir<2>(t, p, a, A, Wau, tau, g, F[2], Ft[2]);
  return ok;
}

}  // namespace dghgks

// Reverse mode (vector-Jacobian products) of the gas-kinetic point fluxes of
// gks_point.cuh: given the cotangents of F and F_t at one face point (or cell
// point), one backward sweep gives the cotangents of the traces (q, dq of
// each side) and of the viscosity.  Every forward intermediate the sweep needs
// is recomputed from the inputs (nothing is stored between points).
//
// Naming: x_b is the cotangent (adjoint) of x; *_b functions accumulate (+=)
// into their cotangent outputs unless stated otherwise.  The functions mirror
// the forward ones statement by statement, in reverse order.
#pragma once

#include "gks_point.cuh"

namespace dghgks {

template <class R>
DG_HD void tab_zero(MomTab<R>& t) {
#pragma unroll
  for (int n = 0; n < 7; ++n) t.u[n] = t.v[n] = t.w[n] = R(0);
  t.xi2 = t.xi4 = R(0);
}

// ---- moment products ----
template <int A, int B, int C, class R>
DG_HD void Gm_b(const MomTab<R>& t, R g, MomTab<R>& tb) {
  tb.u[A] += g * t.v[B] * t.w[C];
  tb.v[B] += g * t.u[A] * t.w[C];
  tb.w[C] += g * t.u[A] * t.v[B];
}
template <int A, int B, int C, class R>
DG_HD void G5_b(const MomTab<R>& t, R g, MomTab<R>& tb) {
  const R h = R(0.5) * g;
  Gm_b<A + 2, B, C>(t, h, tb);
  Gm_b<A, B + 2, C>(t, h, tb);
  Gm_b<A, B, C + 2>(t, h, tb);
  tb.xi2 += h * Gm<A, B, C>(t);
  Gm_b<A, B, C>(t, h * t.xi2, tb);
}
template <int A, int B, int C, class R>
DG_HD void G55_b(const MomTab<R>& t, R g, MomTab<R>& tb) {
  const R q = R(0.25) * g, q2 = R(2) * q;
  Gm_b<A + 4, B, C>(t, q, tb);
  Gm_b<A, B + 4, C>(t, q, tb);
  Gm_b<A, B, C + 4>(t, q, tb);
  Gm_b<A + 2, B + 2, C>(t, q2, tb);
  Gm_b<A + 2, B, C + 2>(t, q2, tb);
  Gm_b<A, B + 2, C + 2>(t, q2, tb);
  tb.xi2 += q2 * (Gm<A + 2, B, C>(t) + Gm<A, B + 2, C>(t) + Gm<A, B, C + 2>(t));
  Gm_b<A + 2, B, C>(t, q2 * t.xi2, tb);
  Gm_b<A, B + 2, C>(t, q2 * t.xi2, tb);
  Gm_b<A, B, C + 2>(t, q2 * t.xi2, tb);
  tb.xi4 += q * Gm<A, B, C>(t);
  Gm_b<A, B, C>(t, q * t.xi4, tb);
}

// KIND 0: Gm, 1: G5, 2: G55
template <int A, int B, int C, int KIND, class R>
DG_HD R gval(const MomTab<R>& t) {
  if constexpr (KIND == 0) return Gm<A, B, C>(t);
  else if constexpr (KIND == 1) return G5<A, B, C>(t);
  else return G55<A, B, C>(t);
}
template <int A, int B, int C, int KIND, class R>
DG_HD void gbar(const MomTab<R>& t, R g, MomTab<R>& tb) {
  if constexpr (KIND == 0) Gm_b<A, B, C>(t, g, tb);
  else if constexpr (KIND == 1) G5_b<A, B, C>(t, g, tb);
  else G55_b<A, B, C>(t, g, tb);
}

// out += s <u^A v^B w^C psi>
template <int A, int B, int C, class R>
DG_HD void mom_psi_b(const MomTab<R>& t, R s, const R ob[5], MomTab<R>& tb, R& sb) {
  sb += ob[0] * Gm<A, B, C>(t) + ob[1] * Gm<A + 1, B, C>(t) + ob[2] * Gm<A, B + 1, C>(t) +
        ob[3] * Gm<A, B, C + 1>(t) + ob[4] * G5<A, B, C>(t);
  Gm_b<A, B, C>(t, s * ob[0], tb);
  Gm_b<A + 1, B, C>(t, s * ob[1], tb);
  Gm_b<A, B + 1, C>(t, s * ob[2], tb);
  Gm_b<A, B, C + 1>(t, s * ob[3], tb);
  G5_b<A, B, C>(t, s * ob[4], tb);
}

// one term out[k] += s a[j] G(t) of mom_a_psi
template <int A, int B, int C, int KIND, class R>
DG_HD void aterm_b(const MomTab<R>& t, const R a[5], R s, const R ob[5], int j, int k, MomTab<R>& tb, R ab[5],
                   R& sb) {
  const R G = gval<A, B, C, KIND>(t);
  ab[j] += s * ob[k] * G;
  sb += ob[k] * a[j] * G;
  gbar<A, B, C, KIND>(t, s * ob[k] * a[j], tb);
}

// out += s <u^A v^B w^C (a . psi) psi>
template <int A, int B, int C, class R>
DG_HD void mom_a_psi_b(const MomTab<R>& t, const R a[5], R s, const R ob[5], MomTab<R>& tb, R ab[5], R& sb) {
  aterm_b<A, B, C, 0>(t, a, s, ob, 0, 0, tb, ab, sb);
  aterm_b<A + 1, B, C, 0>(t, a, s, ob, 1, 0, tb, ab, sb);
  aterm_b<A, B + 1, C, 0>(t, a, s, ob, 2, 0, tb, ab, sb);
  aterm_b<A, B, C + 1, 0>(t, a, s, ob, 3, 0, tb, ab, sb);
  aterm_b<A, B, C, 1>(t, a, s, ob, 4, 0, tb, ab, sb);

  aterm_b<A + 1, B, C, 0>(t, a, s, ob, 0, 1, tb, ab, sb);
  aterm_b<A + 2, B, C, 0>(t, a, s, ob, 1, 1, tb, ab, sb);
  aterm_b<A + 1, B + 1, C, 0>(t, a, s, ob, 2, 1, tb, ab, sb);
  aterm_b<A + 1, B, C + 1, 0>(t, a, s, ob, 3, 1, tb, ab, sb);
  aterm_b<A + 1, B, C, 1>(t, a, s, ob, 4, 1, tb, ab, sb);

  aterm_b<A, B + 1, C, 0>(t, a, s, ob, 0, 2, tb, ab, sb);
  aterm_b<A + 1, B + 1, C, 0>(t, a, s, ob, 1, 2, tb, ab, sb);
  aterm_b<A, B + 2, C, 0>(t, a, s, ob, 2, 2, tb, ab, sb);
  aterm_b<A, B + 1, C + 1, 0>(t, a, s, ob, 3, 2, tb, ab, sb);
  aterm_b<A, B + 1, C, 1>(t, a, s, ob, 4, 2, tb, ab, sb);

  aterm_b<A, B, C + 1, 0>(t, a, s, ob, 0, 3, tb, ab, sb);
  aterm_b<A + 1, B, C + 1, 0>(t, a, s, ob, 1, 3, tb, ab, sb);
  aterm_b<A, B + 1, C + 1, 0>(t, a, s, ob, 2, 3, tb, ab, sb);
  aterm_b<A, B, C + 2, 0>(t, a, s, ob, 3, 3, tb, ab, sb);
  aterm_b<A, B, C + 1, 1>(t, a, s, ob, 4, 3, tb, ab, sb);

  aterm_b<A, B, C, 1>(t, a, s, ob, 0, 4, tb, ab, sb);
  aterm_b<A + 1, B, C, 1>(t, a, s, ob, 1, 4, tb, ab, sb);
  aterm_b<A, B + 1, C, 1>(t, a, s, ob, 2, 4, tb, ab, sb);
  aterm_b<A, B, C + 1, 1>(t, a, s, ob, 3, 4, tb, ab, sb);
  aterm_b<A, B, C, 2>(t, a, s, ob, 4, 4, tb, ab, sb);
}

template <int D, int E, class R>
DG_HD void mom_adotu_psi_b(const MomTab<R>& t, const R a[3][5], R s, const R ob[5], MomTab<R>& tb, R ab[3][5],
                           R& sb) {
  constexpr int A = (D == 0) ? E : 0, B = (D == 1) ? E : 0, C = (D == 2) ? E : 0;
  mom_a_psi_b<A + 1, B, C>(t, a[0], s, ob, tb, ab[0], sb);
  mom_a_psi_b<A, B + 1, C>(t, a[1], s, ob, tb, ab[1], sb);
  mom_a_psi_b<A, B, C + 1>(t, a[2], s, ob, tb, ab[2], sb);
}

// ---- moment tables ----
// tail of the recurrence m[n+2] = U m[n+1] + (n+1) h m[n]
template <class R>
DG_HD void raw_moments_tail_b(const R* m, R U, R h, R* mb, R& Ub, R& hb) {
#pragma unroll
  for (int n = 4; n >= 0; --n) {
    const R g = mb[n + 2];
    Ub += g * m[n + 1];
    mb[n + 1] += g * U;
    hb += g * R(n + 1) * m[n];
    mb[n] += g * R(n + 1) * h;
  }
}

// full line: m[0] = 1, m[1] = U
template <class R>
DG_HD void full_line_b(const R* m, R U, R h, R* mb, R& Ub, R& hb) {
  raw_moments_tail_b(m, U, h, mb, Ub, hb);
  Ub += mb[1];
}

// half line (h = 1 / (2 lam) is passed separately, as in the forward)
template <class R>
DG_HD void half_line_b(const R* m, R U, R lam, R h, int sgn, R* mb, R& Ub, R& lamb, R& hb) {
  raw_moments_tail_b(m, U, h, mb, Ub, hb);
  const R rs = frsqrt(lam);
  const R sl = lam * rs;
  const R ex = fexp(-lam * U * U);
  const R c = R(0.28209479177387814347);  // 1 / (2 sqrt(pi))
  const R e = ex * (c * rs);
  const R sg = sgn > 0 ? R(1) : R(-1);
  // m1 = U m0 + sg e
  Ub += mb[1] * m[0];
  const R m0b = mb[0] + mb[1] * U;
  const R eb = mb[1] * sg;
  // e = exp(-lam U^2) c lam^(-1/2)
  Ub += eb * e * (R(-2) * lam * U);
  lamb += eb * e * (-U * U - R(0.5) / lam);
  // m0 = erfc(-sg sl U) / 2; d erfc(x)/dx = -2/sqrt(pi) exp(-x^2), x^2 = lam U^2
  const R xb = m0b * R(-0.56418958354775628695) * ex;  // -1/sqrt(pi) exp(-x^2)
  // x = -sg sl U, sl = sqrt(lam)
  Ub += xb * (-sg * sl);
  lamb += xb * (-sg * U) * (R(0.5) * rs);
}

template <class R>
DG_HD void full_table_b(const Prim<R>& p, R K, const MomTab<R>& t, MomTab<R>& tb, Prim<R>& pb) {
  const R h = fdiv(R(0.5), p.lam);
  R hb = R(0);
  hb += tb.xi2 * K;
  hb += tb.xi4 * K * (K + R(2)) * R(2) * h;
  full_line_b(t.u, p.U, h, tb.u, pb.U, hb);
  full_line_b(t.v, p.V, h, tb.v, pb.V, hb);
  full_line_b(t.w, p.W, h, tb.w, pb.W, hb);
  pb.lam += hb * (-h / p.lam);  // h = 1/(2 lam)
}

// ---- primitive variables ----
template <class R>
DG_HD void prim_of_b(const R q[5], R gm1, const Prim<R>& p, const Prim<R>& pb, R qb[5]) {
  const R ir = fdiv(R(1), q[0]);
  const R pres = gm1 * (q[4] - R(0.5) * (q[1] * p.U + q[2] * p.V + q[3] * p.W));
  // lam = q0 / (2 pres)
  qb[0] += pb.lam * R(0.5) / pres;
  const R presb = -pb.lam * p.lam / pres;
  // pres = gm1 (q4 - |m|^2 / (2 q0))
  qb[4] += gm1 * presb;
  qb[1] += -gm1 * presb * p.U;
  qb[2] += -gm1 * presb * p.V;
  qb[3] += -gm1 * presb * p.W;
  qb[0] += gm1 * presb * R(0.5) * (p.U * p.U + p.V * p.V + p.W * p.W);
  // U_i = q_i / q0
  qb[1] += pb.U * ir;
  qb[2] += pb.V * ir;
  qb[3] += pb.W * ir;
  qb[0] += -(pb.U * p.U + pb.V * p.V + pb.W * p.W) * ir;
  qb[0] += pb.rho;
}

// ---- slope solve (closed form) ----
template <class R>
DG_HD void slope_solve_b(const Prim<R>& p, R K, const R b[5], const R a[5], const R ab_in[5], Prim<R>& pb,
                         R bb[5]) {
  R ab[5] = {ab_in[0], ab_in[1], ab_in[2], ab_in[3], ab_in[4]};
  const R U[3] = {p.U, p.V, p.W};
  const R E = p.U * p.U + p.V * p.V + p.W * p.W + fdiv((K + R(3)) * R(0.5), p.lam);
  const R r[3] = {b[1] - p.U * b[0], b[2] - p.V * b[0], b[3] - p.W * b[0]};
  const R c4 = fdiv(R(4) * p.lam * p.lam, K + R(3));
  const R X = R(2) * b[4] - E * b[0] - R(2) * (U[0] * r[0] + U[1] * r[1] + U[2] * r[2]);
  const R tl = R(2) * p.lam;
  R Ub[3] = {R(0), R(0), R(0)}, rb[3] = {R(0), R(0), R(0)};
  R Eb = R(0), lamb = R(0);
  // a0 = b0 - U.a[1..3] - a4 E / 2
  bb[0] += ab[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[i] += -ab[0] * a[1 + i];
    ab[1 + i] += -ab[0] * U[i];
  }
  ab[4] += -R(0.5) * ab[0] * E;
  Eb += -R(0.5) * ab[0] * a[4];
  // a_i = tl r_i - U_i a4
  R tlb = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    tlb += ab[1 + i] * r[i];
    rb[i] += ab[1 + i] * tl;
    Ub[i] += -ab[1 + i] * a[4];
    ab[4] += -ab[1 + i] * U[i];
  }
  lamb += R(2) * tlb;
  // a4 = c4 X
  const R Xb = ab[4] * c4;
  lamb += ab[4] * X * fdiv(R(8) * p.lam, K + R(3));
  bb[4] += R(2) * Xb;
  Eb += -Xb * b[0];
  bb[0] += -Xb * E;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[i] += R(-2) * Xb * r[i];
    rb[i] += R(-2) * Xb * U[i];
  }
  // r_i = b_i - U_i b0
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    bb[1 + i] += rb[i];
    Ub[i] += -rb[i] * b[0];
    bb[0] += -rb[i] * U[i];
  }
  // E = |U|^2 + (K+3)/(2 lam)
#pragma unroll
  for (int i = 0; i < 3; ++i) Ub[i] += R(2) * Eb * U[i];
  lamb += -Eb * fdiv((K + R(3)) * R(0.5), p.lam * p.lam);
  pb.U += Ub[0];
  pb.V += Ub[1];
  pb.W += Ub[2];
  pb.lam += lamb;
}

// ---- heat-flux moment ----
template <class R>
DG_HD void heat_of_b(const R F[5], const R W[5], R Un, R Ut1, R Ut2, R Hb, R Fb[5], R Wb[5], R& Unb, R& Ut1b,
                     R& Ut2b) {
  const R U2 = Un * Un + Ut1 * Ut1 + Ut2 * Ut2;
  Fb[4] += Hb;
  Wb[4] += -Hb * Un;
  Unb += -Hb * W[4];
  Fb[1] += -Hb * Un;
  Fb[2] += -Hb * Ut1;
  Fb[3] += -Hb * Ut2;
  Unb += -Hb * F[1];
  Ut1b += -Hb * F[2];
  Ut2b += -Hb * F[3];
  const R S = Un * W[1] + Ut1 * W[2] + Ut2 * W[3];
  Unb += Hb * S;
  Wb[1] += Hb * Un * Un;
  Wb[2] += Hb * Un * Ut1;
  Wb[3] += Hb * Un * Ut2;
  Unb += Hb * Un * W[1];
  Ut1b += Hb * Un * W[2];
  Ut2b += Hb * Un * W[3];
  const R D = F[0] - Un * W[0];
  const R U2b = Hb * R(0.5) * D;
  Fb[0] += Hb * R(0.5) * U2;
  Wb[0] += -Hb * R(0.5) * U2 * Un;
  Unb += -Hb * R(0.5) * U2 * W[0];
  Unb += U2b * R(2) * Un;
  Ut1b += U2b * R(2) * Ut1;
  Ut2b += U2b * R(2) * Ut2;
}

// ---- time-fit weights ----
template <class R>
DG_HD R fit_weights_b(R tau, R dt, R inv_dt, const R wFb[6], const R wFtb[6]) {
  R Eh = R(0), x = R(0);
  const bool pos = tau > R(0);
  if (pos) {
    Eh = fexp(fdiv(R(-0.5) * dt, tau));
    x = tau * inv_dt;
  }
  const R s = R(1) - Eh;
  const R phi = x * s * (R(2) + s);
  const R q = R(4) * x * s * s * inv_dt;
  R taub = R(0), phib = R(0), qb = R(0), sb = R(0);
  // wF
  phib += -wFb[0];
  phib += wFb[1] * R(2) * tau;
  taub += wFb[1] * (R(2) * phi - (R(2) - s * s));
  sb += wFb[1] * tau * R(2) * s;
  phib += wFb[2] * tau;
  taub += wFb[2] * (phi - R(1));
  phib += wFb[3];
  phib += wFb[4] * R(-2) * tau;
  taub += wFb[4] * (R(-2) * phi + R(1) - s * s);
  sb += wFb[4] * tau * R(-2) * s;
  phib += -wFb[5] * tau;
  taub += -wFb[5] * phi;
  // wFt
  qb += wFtb[0];
  qb += wFtb[1] * R(-2) * tau;
  taub += wFtb[1] * R(-2) * q;
  const R esb = wFtb[1] - wFtb[4];
  qb += -wFtb[2] * tau;
  taub += -wFtb[2] * q;
  qb += -wFtb[3];
  qb += wFtb[4] * R(2) * tau;
  taub += wFtb[4] * R(2) * q;
  qb += wFtb[5] * tau;
  taub += wFtb[5] * q;
  if (pos) {
    R xb = R(0), Ehb = R(0);
    // phi = x s (2 + s)
    xb += phib * s * (R(2) + s);
    sb += phib * x * (R(2) + R(2) * s);
    // q = 4 x s^2 / dt
    xb += qb * R(4) * s * s * inv_dt;
    sb += qb * R(8) * x * s * inv_dt;
    // es = 4 x Eh s
    xb += esb * R(4) * Eh * s;
    Ehb += esb * R(4) * x * s;
    sb += esb * R(4) * x * Eh;
    // s = 1 - Eh
    Ehb += -sb;
    taub += xb * inv_dt;
    // Eh = exp(-dt / (2 tau))
    taub += Ehb * Eh * fdiv(R(0.5) * dt, tau * tau);
  }
  return taub;
}

// ---- one side of the interface: cotangents of its sums -> of its traces ----
template <class R>
DG_HD void iface_side_b(int SGN, const R q[5], const R dq[3][5], const GasPar<R>& g, bool pr_fix,
                        const SideSums<R>& Sb, R qb[5], R dqb[3][5]) {
  // forward recomputation
  Prim<R> p;
  prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  R b[3][5], a[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) b[i][k] = dq[i][k] * ir;
    slope_solve(p, g.K, b[i], a[i]);
  }
  MomTab<R> tf;
  full_table(p, g.K, tf);
  R bA[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_adotu_psi<0, 0>(tf, a, R(-1), bA);
  R A[5];
  slope_solve(p, g.K, bA, A);
  MomTab<R> th = tf;
  const R hh = fdiv(R(0.5), p.lam);
  half_line(th.u, p.U, p.lam, hh, SGN);
  const R r = p.rho;

  // backward sweep
  MomTab<R> thb, tfb;
  tab_zero(thb);
  tab_zero(tfb);
  R ab[3][5], Ab[5], rb = R(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Ab[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) ab[i][k] = R(0);
  }
  if (pr_fix) {
    mom_a_psi_b<0, 0, 0>(th, A, r, Sb.W6, thb, Ab, rb);
    mom_adotu_psi_b<0, 0>(th, a, r, Sb.W5, thb, ab, rb);
  }
  mom_a_psi_b<1, 0, 0>(th, A, r, Sb.V6, thb, Ab, rb);
  mom_adotu_psi_b<0, 1>(th, a, r, Sb.V5, thb, ab, rb);
  mom_psi_b<1, 0, 0>(th, r, Sb.V4, thb, rb);
#pragma unroll
  for (int i = 0; i < 3; ++i) mom_a_psi_b<0, 0, 0>(th, a[i], r, Sb.dQ0[i], thb, ab[i], rb);
  mom_psi_b<0, 0, 0>(th, r, Sb.Q0, thb, rb);
  // the half table shares v, w, xi with the full one
  Prim<R> pb;
  pb.rho = rb;
  pb.U = pb.V = pb.W = pb.lam = R(0);
  R hhb = R(0);
  half_line_b(th.u, p.U, p.lam, hh, SGN, thb.u, pb.U, pb.lam, hhb);
  pb.lam += hhb * (-hh / p.lam);
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    tfb.v[n] += thb.v[n];
    tfb.w[n] += thb.w[n];
  }
  tfb.xi2 += thb.xi2;
  tfb.xi4 += thb.xi4;
  // A = solve(bA)
  R bAb[5] = {R(0), R(0), R(0), R(0), R(0)};
  slope_solve_b(p, g.K, bA, A, Ab, pb, bAb);
  // bA = -<(a.u) psi> (full table)
  R sdum = R(0);
  mom_adotu_psi_b<0, 0>(tf, a, R(-1), bAb, tfb, ab, sdum);
  full_table_b(p, g.K, tf, tfb, pb);
  // a_i = solve(dq_i / rho)
  R irb = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R bb[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_b(p, g.K, b[i], a[i], ab[i], pb, bb);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      dqb[i][k] = bb[k] * ir;
      irb += bb[k] * dq[i][k];
    }
  }
  pb.rho += -irb * ir * ir;
#pragma unroll
  for (int k = 0; k < 5; ++k) qb[k] = R(0);
  prim_of_b(q, g.gm1, p, pb, qb);
}

// ---- interface equilibrium and fitted flux: cotangents of F, F_t -> of the sums and mu ----
template <class R>
DG_HD void iface_finish_b(const SideSums<R>& S, const GasPar<R>& g, const R Fb[5], const R Ftb[5], SideSums<R>& Sb,
                          R& mub) {
  const bool pr_fix = (g.pr_fix != R(0));
  // forward recomputation
  Prim<R> p0;
  prim_of(S.Q0, g.gm1, p0);
  const R ir0 = fdiv(R(1), p0.rho);
  R bq[3][5], ab[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) bq[i][k] = S.dQ0[i][k] * ir0;
    slope_solve(p0, g.K, bq[i], ab[i]);
  }
  MomTab<R> t0;
  full_table(p0, g.K, t0);
  R Wab[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_adotu_psi<0, 0>(t0, ab, R(1), Wab);
  R bA[5], Ab[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) bA[k] = -Wab[k];
  slope_solve(p0, g.K, bA, Ab);
  const R tau = fdiv(g.mu * R(2) * p0.lam, p0.rho) + g.tau_add;
  R wF[6], wFt[6];
  fit_weights(tau, g.dt, g.inv_dt, wF, wFt);
  R V1[5] = {R(0), R(0), R(0), R(0), R(0)}, V2[5] = {R(0), R(0), R(0), R(0), R(0)},
    V3[5] = {R(0), R(0), R(0), R(0), R(0)};
  const R r0 = p0.rho;
  mom_psi<1, 0, 0>(t0, r0, V1);
  mom_adotu_psi<0, 1>(t0, ab, r0, V2);
  mom_a_psi<1, 0, 0>(t0, Ab, r0, V3);

  // backward sweep
  R wFb[6], wFtb[6];
  R V1b[5], V2b[5], V3b[5], Wabb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    V1b[k] = V2b[k] = V3b[k] = Wabb[k] = R(0);
    Sb.Q0[k] = Sb.V4[k] = Sb.V5[k] = Sb.V6[k] = Sb.W5[k] = Sb.W6[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) Sb.dQ0[i][k] = R(0);
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) wFb[j] = wFtb[j] = R(0);
  Prim<R> p0b;
  p0b.rho = p0b.U = p0b.V = p0b.W = p0b.lam = R(0);
  R r0b = R(0);
  if (pr_fix) {
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
    const R H[6] = {R(0), H2, H3, H4, H5, H6};  // H[j] pairs with wF[j], wFt[j]
    R Hb[6];
#pragma unroll
    for (int j = 1; j < 6; ++j) {
      Hb[j] = g.pr_fix * (wF[j] * Fb[4] + wFt[j] * Ftb[4]);
      wFb[j] += g.pr_fix * Fb[4] * H[j];
      wFtb[j] += g.pr_fix * Ftb[4] * H[j];
    }
    R W2b[5] = {R(0), R(0), R(0), R(0), R(0)}, W3b[5] = {R(0), R(0), R(0), R(0), R(0)};
    // H[j] is the heat moment weighted by wF[j], wFt[j]: H2 .. H6 for j = 1 .. 5
    heat_of_b(V2, W2, p0.U, p0.V, p0.W, Hb[1], V2b, W2b, p0b.U, p0b.V, p0b.W);
    heat_of_b(V3, W3, p0.U, p0.V, p0.W, Hb[2], V3b, W3b, p0b.U, p0b.V, p0b.W);
    heat_of_b(S.V4, S.Q0, p0.U, p0.V, p0.W, Hb[3], Sb.V4, Sb.Q0, p0b.U, p0b.V, p0b.W);
    heat_of_b(S.V5, S.W5, p0.U, p0.V, p0.W, Hb[4], Sb.V5, Sb.W5, p0b.U, p0b.V, p0b.W);
    heat_of_b(S.V6, S.W6, p0.U, p0.V, p0.W, Hb[5], Sb.V6, Sb.W6, p0b.U, p0b.V, p0b.W);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      Wabb[k] += r0 * (W2b[k] - W3b[k]);
      r0b += Wab[k] * (W2b[k] - W3b[k]);
    }
  }
  // F = sum wF_j V_j, Ft = sum wFt_j V_j
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    wFb[0] += Fb[k] * V1[k];
    wFb[1] += Fb[k] * V2[k];
    wFb[2] += Fb[k] * V3[k];
    wFb[3] += Fb[k] * S.V4[k];
    wFb[4] += Fb[k] * S.V5[k];
    wFb[5] += Fb[k] * S.V6[k];
    wFtb[0] += Ftb[k] * V1[k];
    wFtb[1] += Ftb[k] * V2[k];
    wFtb[2] += Ftb[k] * V3[k];
    wFtb[3] += Ftb[k] * S.V4[k];
    wFtb[4] += Ftb[k] * S.V5[k];
    wFtb[5] += Ftb[k] * S.V6[k];
    V1b[k] += wF[0] * Fb[k] + wFt[0] * Ftb[k];
    V2b[k] += wF[1] * Fb[k] + wFt[1] * Ftb[k];
    V3b[k] += wF[2] * Fb[k] + wFt[2] * Ftb[k];
    Sb.V4[k] += wF[3] * Fb[k] + wFt[3] * Ftb[k];
    Sb.V5[k] += wF[4] * Fb[k] + wFt[4] * Ftb[k];
    Sb.V6[k] += wF[5] * Fb[k] + wFt[5] * Ftb[k];
  }
  MomTab<R> t0b;
  tab_zero(t0b);
  R abb[3][5], Abb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Abb[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) abb[i][k] = R(0);
  }
  mom_a_psi_b<1, 0, 0>(t0, Ab, r0, V3b, t0b, Abb, r0b);
  mom_adotu_psi_b<0, 1>(t0, ab, r0, V2b, t0b, abb, r0b);
  mom_psi_b<1, 0, 0>(t0, r0, V1b, t0b, r0b);
  // tau = 2 mu lam0 / rho0 + tau_add
  const R taub = fit_weights_b(tau, g.dt, g.inv_dt, wFb, wFtb);
  mub += taub * fdiv(R(2) * p0.lam, p0.rho);
  p0b.lam += taub * fdiv(R(2) * g.mu, p0.rho);
  p0b.rho += -taub * fdiv(R(2) * g.mu * p0.lam, p0.rho * p0.rho);
  // Ab = solve(-Wab)
  R bAb[5] = {R(0), R(0), R(0), R(0), R(0)};
  slope_solve_b(p0, g.K, bA, Ab, Abb, p0b, bAb);
#pragma unroll
  for (int k = 0; k < 5; ++k) Wabb[k] += -bAb[k];
  R sdum = R(0);
  mom_adotu_psi_b<0, 0>(t0, ab, R(1), Wabb, t0b, abb, sdum);
  full_table_b(p0, g.K, t0, t0b, p0b);
  p0b.rho += r0b;
  R ir0b = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R bb[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_b(p0, g.K, bq[i], ab[i], abb[i], p0b, bb);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      Sb.dQ0[i][k] += bb[k] * ir0;
      ir0b += bb[k] * S.dQ0[i][k];
    }
  }
  p0b.rho += -ir0b * ir0 * ir0;
  prim_of_b(S.Q0, g.gm1, p0, p0b, Sb.Q0);
}

// VJP of iface_flux: cotangents of (F, F_t) -> of (qL, dqL, qR, dqR) (overwritten) and mu (+=).
template <class R>
DG_HD void iface_flux_vjp(const R qL[5], const R dqL[3][5], const R qR[5], const R dqR[3][5], const GasPar<R>& g,
                          const R Fb[5], const R Ftb[5], R qLb[5], R dqLb[3][5], R qRb[5], R dqRb[3][5], R& mub) {
  const bool pr_fix = (g.pr_fix != R(0));
  SideSums<R> S, Sb;
  iface_zero(S);
  iface_side<R>(1, qL, dqL, g, pr_fix, S);
  iface_side<R>(-1, qR, dqR, g, pr_fix, S);
  iface_finish_b(S, g, Fb, Ftb, Sb, mub);
  iface_side_b<R>(1, qL, dqL, g, pr_fix, Sb, qLb, dqLb);
  iface_side_b<R>(-1, qR, dqR, g, pr_fix, Sb, qRb, dqRb);
}

// ---- interior flux of one direction ----
template <int D, class R>
DG_HD void interior_dir_b(const MomTab<R>& t, const Prim<R>& p, const R a[3][5], const R A[5], const R Wau[5], R tau,
                          const GasPar<R>& g, const R Fb[5], const R Ftb[5], MomTab<R>& tb, Prim<R>& pb,
                          R ab[3][5], R Ab[5], R Waub[5], R& taub) {
  R m0[5] = {R(0), R(0), R(0), R(0), R(0)}, m1[5] = {R(0), R(0), R(0), R(0), R(0)},
    m2[5] = {R(0), R(0), R(0), R(0), R(0)};
  mom_ud_psi<D>(t, R(1), m0);
  mom_adotu_psi<D, 1>(t, a, R(1), m1);
  mom_ud_a_psi<D>(t, A, R(1), m2);
  R m0b[5], m1b[5], m2b[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    // F = rho (m0 - tau (m1 + m2)), Ft = rho m2
    pb.rho += Fb[k] * (m0[k] - tau * (m1[k] + m2[k])) + Ftb[k] * m2[k];
    m0b[k] = Fb[k] * p.rho;
    m1b[k] = -Fb[k] * p.rho * tau;
    m2b[k] = -Fb[k] * p.rho * tau + Ftb[k] * p.rho;
    taub += -Fb[k] * p.rho * (m1[k] + m2[k]);
  }
  if (g.pr_fix != R(0)) {
    const R Un = (D == 0) ? p.U : (D == 1) ? p.V : p.W;
    constexpr int e1 = (D == 0) ? 2 : 1, e2 = (D == 2) ? 2 : 3;
    constexpr int en = 1 + D;
    const int perm[5] = {0, en, e1, e2, 4};
    R Fm1[5], Fm2[5], Wm1[5], Wm2[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      Fm1[k] = m1[perm[k]];
      Fm2[k] = m2[perm[k]];
      Wm1[k] = Wau[perm[k]];
      Wm2[k] = -Wm1[k];
    }
    const R Ut1 = (e1 == 1) ? p.U : (e1 == 2) ? p.V : p.W;
    const R Ut2 = (e2 == 1) ? p.U : (e2 == 2) ? p.V : p.W;
    const R H1 = heat_of(Fm1, Wm1, Un, Ut1, Ut2, 0);
    const R H2 = heat_of(Fm2, Wm2, Un, Ut1, Ut2, 0);
    // F4 += pr rho (-tau (H1 + H2)), Ft4 += pr rho H2
    const R H1b = g.pr_fix * p.rho * (-tau) * Fb[4];
    const R H2b = g.pr_fix * p.rho * ((-tau) * Fb[4] + Ftb[4]);
    pb.rho += g.pr_fix * ((-tau) * (H1 + H2) * Fb[4] + H2 * Ftb[4]);
    taub += -g.pr_fix * p.rho * (H1 + H2) * Fb[4];
    R Fm1b[5] = {R(0), R(0), R(0), R(0), R(0)}, Fm2b[5] = {R(0), R(0), R(0), R(0), R(0)};
    R Wm1b[5] = {R(0), R(0), R(0), R(0), R(0)}, Wm2b[5] = {R(0), R(0), R(0), R(0), R(0)};
    R Unb = R(0), Ut1b = R(0), Ut2b = R(0);
    heat_of_b(Fm1, Wm1, Un, Ut1, Ut2, H1b, Fm1b, Wm1b, Unb, Ut1b, Ut2b);
    heat_of_b(Fm2, Wm2, Un, Ut1, Ut2, H2b, Fm2b, Wm2b, Unb, Ut1b, Ut2b);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      m1b[perm[k]] += Fm1b[k];
      m2b[perm[k]] += Fm2b[k];
      Waub[perm[k]] += Wm1b[k] - Wm2b[k];
    }
    R* Ub[3] = {&pb.U, &pb.V, &pb.W};
    *Ub[D] += Unb;
    *Ub[e1 - 1] += Ut1b;
    *Ub[e2 - 1] += Ut2b;
  }
  R sdum = R(0);
  mom_a_psi_b<(D == 0), (D == 1), (D == 2)>(t, A, R(1), m2b, tb, Ab, sdum);
  mom_adotu_psi_b<D, 1>(t, a, R(1), m1b, tb, ab, sdum);
  mom_psi_b<(D == 0), (D == 1), (D == 2)>(t, R(1), m0b, tb, sdum);
}

// VJP of interior_flux: cotangents of (F[3][5], F_t[3][5]) -> of (q, dq) (overwritten) and mu (+=).
template <class R>
DG_HD void interior_flux_vjp(const R q[5], const R dq[3][5], const GasPar<R>& g, const R Fb[3][5],
                             const R Ftb[3][5], R qb[5], R dqb[3][5], R& mub) {
  Prim<R> p;
  prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  R b[3][5], a[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) b[i][k] = dq[i][k] * ir;
    slope_solve(p, g.K, b[i], a[i]);
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

  MomTab<R> tb;
  tab_zero(tb);
  Prim<R> pb;
  pb.rho = pb.U = pb.V = pb.W = pb.lam = R(0);
  R ab[3][5], Ab[5], Waub[5], taub = R(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Ab[k] = Waub[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) ab[i][k] = R(0);
  }
  interior_dir_b<0>(t, p, a, A, Wau, tau, g, Fb[0], Ftb[0], tb, pb, ab, Ab, Waub, taub);
  interior_dir_b<1>(t, p, a, A, Wau, tau, g, Fb[1], Ftb[1], tb, pb, ab, Ab, Waub, taub);
  interior_dir_b<2>(t, p, a, A, Wau, tau, g, Fb[2], Ftb[2], tb, pb, ab, Ab, Waub, taub);
  // tau = 2 mu lam / rho + tau_add
  mub += taub * fdiv(R(2) * p.lam, p.rho);
  pb.lam += taub * fdiv(R(2) * g.mu, p.rho);
  pb.rho += -taub * fdiv(R(2) * g.mu * p.lam, p.rho * p.rho);
  // A = solve(-Wau)
  R bAb[5] = {R(0), R(0), R(0), R(0), R(0)};
  slope_solve_b(p, g.K, bA, A, Ab, pb, bAb);
#pragma unroll
  for (int k = 0; k < 5; ++k) Waub[k] += -bAb[k];
  R sdum = R(0);
  mom_adotu_psi_b<0, 0>(t, a, R(1), Waub, tb, ab, sdum);
  full_table_b(p, g.K, t, tb, pb);
  R irb = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R bb[5] = {R(0), R(0), R(0), R(0), R(0)};
    slope_solve_b(p, g.K, b[i], a[i], ab[i], pb, bb);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      dqb[i][k] = bb[k] * ir;
      irb += bb[k] * dq[i][k];
    }
  }
  pb.rho += -irb * ir * ir;
#pragma unroll
  for (int k = 0; k < 5; ++k) qb[k] = R(0);
  prim_of_b(q, g.gm1, p, pb, qb);
}

}  // namespace dghgks

// Reverse mode (vector-Jacobian products) of the gas-kinetic point fluxes of
// gks_point.cuh: given the cotangents of F and F_t at one face point (or cell
// point), one backward sweep gives the cotangents of the traces (q, dq of
// each side) and of the viscosity.  Every forward intermediate the sweep needs
// is recomputed from the inputs (nothing is stored between points).  The
// sweeps follow the forward's formulation: moments in the frame of each
// Maxwellian, parity-sparse moment contractions, frame shifts.
//
// Naming: x_b is the cotangent (adjoint) of x; *_b functions accumulate (+=)
// into their cotangent outputs unless stated otherwise.  The functions mirror
// the forward ones statement by statement, in reverse order.
#pragma once

#include "gks_point.cuh"

namespace dghgks {

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


// ---- frame-centred moment tables ----
template <class R>
struct CTabB {  // cotangent of a CTab
  R u[7];
  R c2, c4, c6, xi2, xi4;
};
template <class R>
DG_HD void ctab_zero(CTabB<R>& b) {
#pragma unroll
  for (int n = 0; n < 7; ++n) b.u[n] = R(0);
  b.c2 = b.c4 = b.c6 = b.xi2 = b.xi4 = R(0);
}
template <int N, class R>
DG_HD R& cm_c_b(CTabB<R>& tb) {
  static_assert(N == 2 || N == 4 || N == 6, "central moment cotangent");
  if constexpr (N == 2) return tb.c2;
  else if constexpr (N == 4) return tb.c4;
  else return tb.c6;
}
// cm = x_A c_B c_C (x_A = t.u[A], or the central moment when CU; power-0 factors are 1)
template <bool CU, int A, int B, int C, class R>
DG_HD void cm_b(const CTab<R>& t, R g, CTabB<R>& tb) {
  R fa;
  if constexpr (CU) fa = cm_c<A>(t);
  else fa = t.u[A];
  const R fb = cm_c<B>(t), fc = cm_c<C>(t);
  if constexpr (CU) {
    if constexpr (A > 0) cm_c_b<A>(tb) += g * fb * fc;
  } else {
    tb.u[A] += g * fb * fc;
  }
  if constexpr (B > 0) cm_c_b<B>(tb) += g * fa * fc;
  if constexpr (C > 0) cm_c_b<C>(tb) += g * fa * fb;
}
template <bool CU, int A, int B, int C, class R>
DG_HD void cm5_b(const CTab<R>& t, R g, CTabB<R>& tb) {
  const R h = R(0.5) * g;
  cm_b<CU, A + 2, B, C>(t, h, tb);
  cm_b<CU, A, B + 2, C>(t, h, tb);
  cm_b<CU, A, B, C + 2>(t, h, tb);
  tb.xi2 += h * cm<CU, A, B, C>(t);
  cm_b<CU, A, B, C>(t, h * t.xi2, tb);
}
template <bool CU, int A, int B, int C, class R>
DG_HD void cm55_b(const CTab<R>& t, R g, CTabB<R>& tb) {
  const R q = R(0.25) * g, q2 = R(2) * q;
  cm_b<CU, A + 4, B, C>(t, q, tb);
  cm_b<CU, A, B + 4, C>(t, q, tb);
  cm_b<CU, A, B, C + 4>(t, q, tb);
  cm_b<CU, A + 2, B + 2, C>(t, q2, tb);
  cm_b<CU, A + 2, B, C + 2>(t, q2, tb);
  cm_b<CU, A, B + 2, C + 2>(t, q2, tb);
  tb.xi2 += q2 * (cm<CU, A + 2, B, C>(t) + cm<CU, A, B + 2, C>(t) + cm<CU, A, B, C + 2>(t));
  cm_b<CU, A + 2, B, C>(t, q2 * t.xi2, tb);
  cm_b<CU, A, B + 2, C>(t, q2 * t.xi2, tb);
  cm_b<CU, A, B, C + 2>(t, q2 * t.xi2, tb);
  tb.xi4 += q * cm<CU, A, B, C>(t);
  cm_b<CU, A, B, C>(t, q * t.xi4, tb);
}
template <bool CU, int J, int K, int A, int B, int C, class R>
DG_HD void ent_b(const CTab<R>& t, R g, CTabB<R>& tb) {
  if constexpr (J == 4 && K == 4) cm55_b<CU, A, B, C>(t, g, tb);
  else if constexpr (J == 4) cm5_b<CU, A + (K == 1), B + (K == 2), C + (K == 3)>(t, g, tb);
  else if constexpr (K == 4) cm5_b<CU, A + (J == 1), B + (J == 2), C + (J == 3)>(t, g, tb);
  else cm_b<CU, A + (J == 1) + (K == 1), B + (J == 2) + (K == 2), C + (J == 3) + (K == 3)>(t, g, tb);
}
// reverse of out += <c^ABC (a . psi') psi'>: ab += d/da, tb += d/dt
template <bool CU, int A, int B, int C, int K, int J, class R>
DG_HD void cmom_a_term_b(const CTab<R>& t, const R a[5], const R ob[5], CTabB<R>& tb, R ab[5]) {
  if constexpr (!ent_zero<CU, J, K, A, B, C>()) {
    ab[J] += ob[K] * ent<CU, J, K, A, B, C>(t);
    ent_b<CU, J, K, A, B, C>(t, ob[K] * a[J], tb);
  }
}
template <bool CU, int A, int B, int C, class R, int... I>
DG_HD void cmom_a_seq_b(const CTab<R>& t, const R a[5], const R ob[5], CTabB<R>& tb, R ab[5],
                        std::integer_sequence<int, I...>) {
  (cmom_a_term_b<CU, A, B, C, I / 5, I % 5>(t, a, ob, tb, ab), ...);
}
template <bool CU, int A, int B, int C, class R>
DG_HD void cmom_a_b(const CTab<R>& t, const R a[5], const R ob[5], CTabB<R>& tb, R ab[5]) {
  cmom_a_seq_b<CU, A, B, C>(t, a, ob, tb, ab, std::make_integer_sequence<int, 25>{});
}
template <bool CU, int D, class R>
DG_HD void cmom_a_e_b(const CTab<R>& t, const R a[5], const R ob[5], CTabB<R>& tb, R ab[5]) {
  cmom_a_b<CU, D == 0, D == 1, D == 2>(t, a, ob, tb, ab);
}
template <bool CU, int D, int E, class R>
DG_HD void cmom_a_ee_b(const CTab<R>& t, const R a[5], const R ob[5], CTabB<R>& tb, R ab[5]) {
  cmom_a_b<CU, (D == 0) + (E == 0), (D == 1) + (E == 1), (D == 2) + (E == 2)>(t, a, ob, tb, ab);
}
// reverse of out += s <c^ABC psi'>
template <bool CU, int A, int B, int C, int K, class R>
DG_HD void cmom_psi_term_b(const CTab<R>& t, R s, const R ob[5], CTabB<R>& tb, R& sb) {
  if constexpr (!ent_zero<CU, 0, K, A, B, C>()) {
    sb += ob[K] * ent<CU, 0, K, A, B, C>(t);
    ent_b<CU, 0, K, A, B, C>(t, s * ob[K], tb);
  }
}
template <bool CU, int A, int B, int C, class R>
DG_HD void cmom_psi_b(const CTab<R>& t, R s, const R ob[5], CTabB<R>& tb, R& sb) {
  cmom_psi_term_b<CU, A, B, C, 0>(t, s, ob, tb, sb);
  cmom_psi_term_b<CU, A, B, C, 1>(t, s, ob, tb, sb);
  cmom_psi_term_b<CU, A, B, C, 2>(t, s, ob, tb, sb);
  cmom_psi_term_b<CU, A, B, C, 3>(t, s, ob, tb, sb);
  cmom_psi_term_b<CU, A, B, C, 4>(t, s, ob, tb, sb);
}
// reverse of cent_table: returns the cotangent of h
template <class R>
DG_HD R cent_table_b(R h, R K, const CTabB<R>& tb) {
  return tb.c2 + tb.c4 * R(6) * h + tb.c6 * R(45) * h * h + tb.xi2 * K + tb.xi4 * R(2) * K * (K + R(2)) * h;
}

// ---- frame shifts ----
template <class R>
DG_HD void to_centred_b(const R m[5], R U, R V, R W, R hs2, const R ob[5], R mb[5], R& Ub, R& Vb, R& Wb, R& hs2b) {
  mb[0] += ob[0] - U * ob[1] - V * ob[2] - W * ob[3] + hs2 * ob[4];
  mb[1] += ob[1] - U * ob[4];
  mb[2] += ob[2] - V * ob[4];
  mb[3] += ob[3] - W * ob[4];
  mb[4] += ob[4];
  Ub += -ob[1] * m[0] - ob[4] * m[1];
  Vb += -ob[2] * m[0] - ob[4] * m[2];
  Wb += -ob[3] * m[0] - ob[4] * m[3];
  hs2b += ob[4] * m[0];
}
template <bool SU, class R>
DG_HD void add_uncentred_b(const R mp[5], R U, R V, R W, R hs2, const R ob[5], R mpb[5], R& Ub, R& Vb, R& Wb,
                           R& hs2b) {
  mpb[0] += ob[0] + V * ob[2] + W * ob[3] + hs2 * ob[4];
  mpb[1] += ob[1];
  if constexpr (SU) {
    mpb[0] += U * ob[1];
    mpb[1] += U * ob[4];
    Ub += ob[1] * mp[0] + ob[4] * mp[1];
  }
  mpb[2] += ob[2] + V * ob[4];
  mpb[3] += ob[3] + W * ob[4];
  mpb[4] += ob[4];
  Vb += ob[2] * mp[0] + ob[4] * mp[2];
  Wb += ob[3] * mp[0] + ob[4] * mp[3];
  hs2b += ob[4] * mp[0];
}
// component 4 of to_centred (the heat-moment part)
template <class R>
DG_HD R cen4(const R m[5], R U, R V, R W, R hs2) {
  return m[4] - U * m[1] - V * m[2] - W * m[3] + hs2 * m[0];
}
template <class R>
DG_HD void cen4_b(const R m[5], R U, R V, R W, R hs2, R g, R mb[5], R& Ub, R& Vb, R& Wb, R& hs2b) {
  mb[4] += g;
  mb[1] += -U * g;
  mb[2] += -V * g;
  mb[3] += -W * g;
  mb[0] += hs2 * g;
  Ub += -g * m[1];
  Vb += -g * m[2];
  Wb += -g * m[3];
  hs2b += g * m[0];
}
// reverse of coef_shift_u (a = the coefficients before the shift; ab: cotangent
// of the shifted ones on entry, of the unshifted ones on exit)
template <class R>
DG_HD void coef_shift_u_b(const R a[5], R d, R ab[5], R& db) {
  const R a0b = ab[0], a1b = ab[1];
  db += a0b * (a[1] + d * a[4]) + a1b * a[4];
  ab[1] = a1b + a0b * d;
  ab[4] += a0b * R(0.5) * d * d + a1b * d;
  ab[0] = a0b;
}

// ---- centred slope solves ----
template <class R>
struct CSolveB {
  R e1, k4, tlam;
};
template <class R>
DG_HD void centred_solver_b(R lam, R h, R K, const CSolveB<R>& csb, R& lamb, R& hb) {
  hb += csb.e1 * R(0.5) * (K + R(3));
  lamb += csb.k4 * fdiv(R(16) * lam, K + R(3)) + R(2) * csb.tlam;
}
template <class R>
DG_HD void centred_solve_b(const CSolve<R>& cs, const R b[5], const R a[5], const R ab[5], R bb[5], CSolveB<R>& csb) {
  R a4b = ab[4];
  // a0 = b0 - e1 a4
  bb[0] += ab[0];
  csb.e1 += -ab[0] * a[4];
  a4b += -ab[0] * cs.e1;
  // a_i = tlam b_i
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    csb.tlam += ab[i] * b[i];
    bb[i] += ab[i] * cs.tlam;
  }
  // a4 = k4 (b4 - e1 b0)
  csb.k4 += a4b * (b[4] - cs.e1 * b[0]);
  bb[4] += a4b * cs.k4;
  bb[0] += -a4b * cs.k4 * cs.e1;
  csb.e1 += -a4b * cs.k4 * b[0];
}
// Reverse of centred_slopes: ab, Waub, Ab are the cotangents of a_i, Wau, A
// (ab is consumed); adds to dqb, irb, the velocity and hs2 cotangents, tb, csb.
template <class R>
DG_HD void centred_slopes_b(const Prim<R>& p, R ir, R hs2, const CSolve<R>& cs, const CTab<R>& t, const R dq[3][5],
                            R ab[3][5], const R Waub[5], const R Ab[5], R dqb[3][5], R& irb, Prim<R>& pb, R& hs2b,
                            CTabB<R>& tb, CSolveB<R>& csb) {
  // forward recomputation
  const R Uc[3] = {p.U, p.V, p.W};
  R b[3][5], bc[3][5], a[3][5], Wau[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) b[i][k] = dq[i][k] * ir;
    to_centred(b[i], p.U, p.V, p.W, hs2, bc[i]);
    centred_solve(cs, bc[i], a[i]);
#pragma unroll
    for (int k = 0; k < 5; ++k) Wau[k] += Uc[i] * bc[i][k];
  }
  cmom_a_e<true, 0>(t, a[0], Wau);
  cmom_a_e<true, 1>(t, a[1], Wau);
  cmom_a_e<true, 2>(t, a[2], Wau);
  R bA[5], A[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) bA[k] = -Wau[k];
  centred_solve(cs, bA, A);
  // A = solve(-Wau)
  R bAb[5] = {R(0), R(0), R(0), R(0), R(0)};
  centred_solve_b(cs, bA, A, Ab, bAb, csb);
  R Wb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Wb[k] = Waub[k] - bAb[k];
  // Wau = sum_i U_i bc_i + sum_i <c_i (a_i . psi'') psi''>
  cmom_a_e_b<true, 0>(t, a[0], Wb, tb, ab[0]);
  cmom_a_e_b<true, 1>(t, a[1], Wb, tb, ab[1]);
  cmom_a_e_b<true, 2>(t, a[2], Wb, tb, ab[2]);
  R Ub[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R bcb[5], bb[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      bcb[k] = Uc[i] * Wb[k];
      Ub[i] += Wb[k] * bc[i][k];
    }
    centred_solve_b(cs, bc[i], a[i], ab[i], bcb, csb);
    to_centred_b(b[i], p.U, p.V, p.W, hs2, bcb, bb, Ub[0], Ub[1], Ub[2], hs2b);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      dqb[i][k] += bb[k] * ir;
      irb += bb[k] * dq[i][k];
    }
  }
  pb.U += Ub[0];
  pb.V += Ub[1];
  pb.W += Ub[2];
}

// ---- one side of the interface: cotangents of its sums -> of its traces ----
template <class R>
DG_HD void iface_side_b(int SGN, const R q[5], const R dq[3][5], const GasPar<R>& g, bool pr_fix,
                        const SideSums<R>& Sb, R qb[5], R dqb[3][5]) {
  // forward recomputation (iface_side)
  Prim<R> p;
  prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  const R h = fdiv(R(0.5), p.lam);
  const R ht2 = R(0.5) * (p.V * p.V + p.W * p.W);
  const R hs2 = R(0.5) * p.U * p.U + ht2;
  CTab<R> t;
  cent_table(h, g.K, t);
  CSolve<R> cs;
  centred_solver(p.lam, h, g.K, cs);
  R a[3][5], Wau[5], A[5];
  centred_slopes(p, ir, hs2, cs, t, dq, a, Wau, A);
  const R r = p.rho, d = -p.U;
  R a1[3][5], A1[5], as[3][5], As[5], aVW[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) A1[k] = A[k];
  coef_shift_u(A1, d);
#pragma unroll
  for (int k = 0; k < 5; ++k) As[k] = r * A1[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) a1[i][k] = a[i][k];
    coef_shift_u(a1[i], d);
#pragma unroll
    for (int k = 0; k < 5; ++k) as[i][k] = r * a1[i][k];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) aVW[k] = p.V * as[1][k] + p.W * as[2][k];
  half_line(t.u, p.U, p.lam, h, SGN);
  R mQ0[5], mdQ0[3][5], mV4[5], mV5[5], mV6[5], mW5[5], mW6[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    mQ0[k] = mV4[k] = mV5[k] = mV6[k] = mW5[k] = mW6[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) mdQ0[i][k] = R(0);
  }
  cmom_psi<false, 0, 0, 0>(t, r, mQ0);
#pragma unroll
  for (int i = 0; i < 3; ++i) cmom_a<false, 0, 0, 0>(t, as[i], mdQ0[i]);
  cmom_psi<false, 1, 0, 0>(t, r, mV4);
  cmom_a<false, 2, 0, 0>(t, as[0], mV5);
  cmom_a<false, 1, 1, 0>(t, as[1], mV5);
  cmom_a<false, 1, 0, 1>(t, as[2], mV5);
  cmom_a<false, 1, 0, 0>(t, aVW, mV5);
  cmom_a<false, 1, 0, 0>(t, As, mV6);
  if (pr_fix) {
    cmom_a<false, 1, 0, 0>(t, as[0], mW5);
    cmom_a<false, 0, 1, 0>(t, as[1], mW5);
    cmom_a<false, 0, 0, 1>(t, as[2], mW5);
    cmom_a<false, 0, 0, 0>(t, aVW, mW5);
    cmom_a<false, 0, 0, 0>(t, As, mW6);
  }

  // backward sweep
  R Vb = R(0), Wb = R(0), ht2b = R(0), rb = R(0), Udum = R(0);
  CTabB<R> tb;
  ctab_zero(tb);
  R asb[3][5], Asb[5], aVWb[5], mb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Asb[k] = aVWb[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) asb[i][k] = R(0);
  }
  // each sum: out += S_(0,V,W) m  ->  mb
  auto unshift_b = [&](const R m[5], const R ob[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) mb[k] = R(0);
    add_uncentred_b<false>(m, R(0), p.V, p.W, ht2, ob, mb, Udum, Vb, Wb, ht2b);
  };
  if (pr_fix) {
    unshift_b(mW6, Sb.W6);
    cmom_a_b<false, 0, 0, 0>(t, As, mb, tb, Asb);
    unshift_b(mW5, Sb.W5);
    cmom_a_b<false, 1, 0, 0>(t, as[0], mb, tb, asb[0]);
    cmom_a_b<false, 0, 1, 0>(t, as[1], mb, tb, asb[1]);
    cmom_a_b<false, 0, 0, 1>(t, as[2], mb, tb, asb[2]);
    cmom_a_b<false, 0, 0, 0>(t, aVW, mb, tb, aVWb);
  }
  unshift_b(mV6, Sb.V6);
  cmom_a_b<false, 1, 0, 0>(t, As, mb, tb, Asb);
  unshift_b(mV5, Sb.V5);
  cmom_a_b<false, 2, 0, 0>(t, as[0], mb, tb, asb[0]);
  cmom_a_b<false, 1, 1, 0>(t, as[1], mb, tb, asb[1]);
  cmom_a_b<false, 1, 0, 1>(t, as[2], mb, tb, asb[2]);
  cmom_a_b<false, 1, 0, 0>(t, aVW, mb, tb, aVWb);
  unshift_b(mV4, Sb.V4);
  cmom_psi_b<false, 1, 0, 0>(t, r, mb, tb, rb);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    unshift_b(mdQ0[i], Sb.dQ0[i]);
    cmom_a_b<false, 0, 0, 0>(t, as[i], mb, tb, asb[i]);
  }
  unshift_b(mQ0, Sb.Q0);
  cmom_psi_b<false, 0, 0, 0>(t, r, mb, tb, rb);
  // aVW = V as_1 + W as_2
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    asb[1][k] += p.V * aVWb[k];
    asb[2][k] += p.W * aVWb[k];
    Vb += aVWb[k] * as[1][k];
    Wb += aVWb[k] * as[2][k];
  }
  // half-space line (the centred uses above read only the central moments)
  Prim<R> pb;
  pb.rho = pb.U = pb.V = pb.W = pb.lam = R(0);
  R hb = R(0);
  half_line_b(t.u, p.U, p.lam, h, SGN, tb.u, pb.U, pb.lam, hb);
  // as = r a1, As = r A1; a1 = shift(a, -U), A1 = shift(A, -U)
  R db = R(0), Ab[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    rb += Asb[k] * A1[k];
    Ab[k] = r * Asb[k];
  }
  coef_shift_u_b(A, d, Ab, db);
  R ab[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      rb += asb[i][k] * a1[i][k];
      ab[i][k] = r * asb[i][k];
    }
    coef_shift_u_b(a[i], d, ab[i], db);
  }
  pb.U += -db;
  // slopes and compatibility
  const R Waub0[5] = {R(0), R(0), R(0), R(0), R(0)};
  R irb = R(0), hs2b = R(0);
  CSolveB<R> csb;
  csb.e1 = csb.k4 = csb.tlam = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 5; ++k) dqb[i][k] = R(0);
  centred_slopes_b(p, ir, hs2, cs, t, dq, ab, Waub0, Ab, dqb, irb, pb, hs2b, tb, csb);
  // tables
  centred_solver_b(p.lam, h, g.K, csb, pb.lam, hb);
  hb += cent_table_b(h, g.K, tb);
  pb.lam += hb * (-h / p.lam);  // h = 1/(2 lam)
  // hs2 = U^2/2 + ht2, ht2 = (V^2 + W^2)/2
  pb.U += hs2b * p.U;
  ht2b += hs2b;
  pb.V += ht2b * p.V + Vb;
  pb.W += ht2b * p.W + Wb;
  pb.rho += rb - irb * ir * ir;
#pragma unroll
  for (int k = 0; k < 5; ++k) qb[k] = R(0);
  prim_of_b(q, g.gm1, p, pb, qb);
}

// ---- interface equilibrium and fitted flux: cotangents of F, F_t -> of the sums and mu ----
// FTO: the cotangent of F is zero (stage 2 of the S2O4 adjoint, where only
// L_t enters): Fb is not read, and F, the heat-flux term (F only) and every
// product with the zero cotangent are left out of both sweeps.
template <class R, bool FTO = false>
DG_HD void iface_finish_b(const SideSums<R>& S, const GasPar<R>& g, const R Fb[5], const R Ftb[5], SideSums<R>& Sb,
                          R& mub) {
  const bool pr_fix = !FTO && (g.pr_fix != R(0));
  // forward recomputation (iface_finish)
  Prim<R> p0;
  prim_of(S.Q0, g.gm1, p0);
  const R ir0 = fdiv(R(1), p0.rho);
  const R h = fdiv(R(0.5), p0.lam);
  const R U = p0.U, V = p0.V, W = p0.W;
  const R hs2 = R(0.5) * (U * U + V * V + W * W);
  CTab<R> t0;
  cent_table(h, g.K, t0);
  CSolve<R> cs;
  centred_solver(p0.lam, h, g.K, cs);
  R ab[3][5], Wab[5], Ab[5];
  centred_slopes(p0, ir0, hs2, cs, t0, S.dQ0, ab, Wab, Ab);
  const R tau = fdiv(g.mu * R(2) * p0.lam, p0.rho) + g.tau_add;
  R wF[6], wFt[6];
  fit_weights(tau, g.dt, g.inv_dt, wF, wFt);
  R V1[5] = {R(0), R(0), R(0), R(0), R(0)}, V2[5], V3[5], aU[5];
  cmom_psi<true, 0, 0, 0>(t0, U, V1);
  cmom_psi<true, 1, 0, 0>(t0, R(1), V1);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    aU[k] = U * ab[0][k] + V * ab[1][k] + W * ab[2][k];
    V2[k] = U * Wab[k];
    V3[k] = -U * Wab[k];
  }
  cmom_a_ee<true, 0, 0>(t0, ab[0], V2);
  cmom_a_ee<true, 0, 1>(t0, ab[1], V2);
  cmom_a_ee<true, 0, 2>(t0, ab[2], V2);
  cmom_a_e<true, 0>(t0, aU, V2);
  cmom_a_e<true, 0>(t0, Ab, V3);
  R V4[5], V5[5], V6[5];
  to_centred(S.V4, U, V, W, hs2, V4);
  to_centred(S.V5, U, V, W, hs2, V5);
  to_centred(S.V6, U, V, W, hs2, V6);
  const R r0 = p0.rho;
  R Fc[5], Ftc[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (!FTO)
      Fc[k] = r0 * (wF[0] * V1[k] + wF[1] * V2[k] + wF[2] * V3[k]) + wF[3] * V4[k] + wF[4] * V5[k] + wF[5] * V6[k];
    Ftc[k] = r0 * (wFt[0] * V1[k] + wFt[1] * V2[k] + wFt[2] * V3[k]) + wFt[3] * V4[k] + wFt[4] * V5[k] +
             wFt[5] * V6[k];
  }
  R H[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (pr_fix) {
    H[1] = r0 * (V2[4] - U * Wab[4]);
    H[2] = r0 * (V3[4] + U * Wab[4]);
    H[3] = V4[4] - U * cen4(S.Q0, U, V, W, hs2);
    H[4] = V5[4] - U * cen4(S.W5, U, V, W, hs2);
    H[5] = V6[4] - U * cen4(S.W6, U, V, W, hs2);
    Fc[4] += g.pr_fix * (wF[1] * H[1] + wF[2] * H[2] + wF[3] * H[3] + wF[4] * H[4] + wF[5] * H[5]);
  }

  // backward sweep
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Sb.Q0[k] = Sb.V4[k] = Sb.V5[k] = Sb.V6[k] = Sb.W5[k] = Sb.W6[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) Sb.dQ0[i][k] = R(0);
  }
  Prim<R> p0b;
  p0b.rho = p0b.U = p0b.V = p0b.W = p0b.lam = R(0);
  R hs2b = R(0), r0b = R(0), wFb[6], wFtb[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) wFb[j] = wFtb[j] = R(0);
  // F = S_U Fc, Ft = S_U Ftc
  R Fcb[5] = {R(0), R(0), R(0), R(0), R(0)}, Ftcb[5] = {R(0), R(0), R(0), R(0), R(0)};
  if (!FTO) add_uncentred_b<true>(Fc, U, V, W, hs2, Fb, Fcb, p0b.U, p0b.V, p0b.W, hs2b);
  add_uncentred_b<true>(Ftc, U, V, W, hs2, Ftb, Ftcb, p0b.U, p0b.V, p0b.W, hs2b);
  R V1b[5], V2b[5], V3b[5], V4b[5], V5b[5], V6b[5], Wabb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) V1b[k] = V2b[k] = V3b[k] = V4b[k] = V5b[k] = V6b[k] = Wabb[k] = R(0);
  if (pr_fix) {
    R Hb[6];
#pragma unroll
    for (int j = 1; j < 6; ++j) {
      Hb[j] = g.pr_fix * wF[j] * Fcb[4];
      wFb[j] += g.pr_fix * Fcb[4] * H[j];
    }
    r0b += Hb[1] * (V2[4] - U * Wab[4]) + Hb[2] * (V3[4] + U * Wab[4]);
    V2b[4] += Hb[1] * r0;
    V3b[4] += Hb[2] * r0;
    p0b.U += (Hb[2] - Hb[1]) * r0 * Wab[4];
    Wabb[4] += (Hb[2] - Hb[1]) * r0 * U;
    V4b[4] += Hb[3];
    V5b[4] += Hb[4];
    V6b[4] += Hb[5];
    p0b.U += -Hb[3] * cen4(S.Q0, U, V, W, hs2) - Hb[4] * cen4(S.W5, U, V, W, hs2) - Hb[5] * cen4(S.W6, U, V, W, hs2);
    cen4_b(S.Q0, U, V, W, hs2, -Hb[3] * U, Sb.Q0, p0b.U, p0b.V, p0b.W, hs2b);
    cen4_b(S.W5, U, V, W, hs2, -Hb[4] * U, Sb.W5, p0b.U, p0b.V, p0b.W, hs2b);
    cen4_b(S.W6, U, V, W, hs2, -Hb[5] * U, Sb.W6, p0b.U, p0b.V, p0b.W, hs2b);
  }
  // Fc = r0 (wF0 V1 + wF1 V2 + wF2 V3) + wF3 V4 + wF4 V5 + wF5 V6, Ftc alike
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if constexpr (FTO) {
      r0b += Ftcb[k] * (wFt[0] * V1[k] + wFt[1] * V2[k] + wFt[2] * V3[k]);
      wFtb[0] += Ftcb[k] * r0 * V1[k];
      wFtb[1] += Ftcb[k] * r0 * V2[k];
      wFtb[2] += Ftcb[k] * r0 * V3[k];
      wFtb[3] += Ftcb[k] * V4[k];
      wFtb[4] += Ftcb[k] * V5[k];
      wFtb[5] += Ftcb[k] * V6[k];
      V1b[k] += r0 * (wFt[0] * Ftcb[k]);
      V2b[k] += r0 * (wFt[1] * Ftcb[k]);
      V3b[k] += r0 * (wFt[2] * Ftcb[k]);
      V4b[k] += wFt[3] * Ftcb[k];
      V5b[k] += wFt[4] * Ftcb[k];
      V6b[k] += wFt[5] * Ftcb[k];
      continue;
    }
    r0b += Fcb[k] * (wF[0] * V1[k] + wF[1] * V2[k] + wF[2] * V3[k]) +
           Ftcb[k] * (wFt[0] * V1[k] + wFt[1] * V2[k] + wFt[2] * V3[k]);
    wFb[0] += Fcb[k] * r0 * V1[k];
    wFb[1] += Fcb[k] * r0 * V2[k];
    wFb[2] += Fcb[k] * r0 * V3[k];
    wFb[3] += Fcb[k] * V4[k];
    wFb[4] += Fcb[k] * V5[k];
    wFb[5] += Fcb[k] * V6[k];
    wFtb[0] += Ftcb[k] * r0 * V1[k];
    wFtb[1] += Ftcb[k] * r0 * V2[k];
    wFtb[2] += Ftcb[k] * r0 * V3[k];
    wFtb[3] += Ftcb[k] * V4[k];
    wFtb[4] += Ftcb[k] * V5[k];
    wFtb[5] += Ftcb[k] * V6[k];
    V1b[k] += r0 * (wF[0] * Fcb[k] + wFt[0] * Ftcb[k]);
    V2b[k] += r0 * (wF[1] * Fcb[k] + wFt[1] * Ftcb[k]);
    V3b[k] += r0 * (wF[2] * Fcb[k] + wFt[2] * Ftcb[k]);
    V4b[k] += wF[3] * Fcb[k] + wFt[3] * Ftcb[k];
    V5b[k] += wF[4] * Fcb[k] + wFt[4] * Ftcb[k];
    V6b[k] += wF[5] * Fcb[k] + wFt[5] * Ftcb[k];
  }
  to_centred_b(S.V4, U, V, W, hs2, V4b, Sb.V4, p0b.U, p0b.V, p0b.W, hs2b);
  to_centred_b(S.V5, U, V, W, hs2, V5b, Sb.V5, p0b.U, p0b.V, p0b.W, hs2b);
  to_centred_b(S.V6, U, V, W, hs2, V6b, Sb.V6, p0b.U, p0b.V, p0b.W, hs2b);
  CTabB<R> t0b;
  ctab_zero(t0b);
  R abb[3][5], Abb[5], aUb[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Abb[k] = aUb[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) abb[i][k] = R(0);
  }
  // V3 = -U Wab + <c_u (Abar . psi'') psi''>
  cmom_a_e_b<true, 0>(t0, Ab, V3b, t0b, Abb);
  // V2 = U Wab + sum_i <c_u c_i (abar_i . psi'') psi''> + <c_u (aU . psi'') psi''>
  cmom_a_e_b<true, 0>(t0, aU, V2b, t0b, aUb);
  cmom_a_ee_b<true, 0, 2>(t0, ab[2], V2b, t0b, abb[2]);
  cmom_a_ee_b<true, 0, 1>(t0, ab[1], V2b, t0b, abb[1]);
  cmom_a_ee_b<true, 0, 0>(t0, ab[0], V2b, t0b, abb[0]);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    p0b.U += (V2b[k] - V3b[k]) * Wab[k];
    Wabb[k] += U * (V2b[k] - V3b[k]);
    // aU = U ab_0 + V ab_1 + W ab_2
    abb[0][k] += U * aUb[k];
    abb[1][k] += V * aUb[k];
    abb[2][k] += W * aUb[k];
    p0b.U += aUb[k] * ab[0][k];
    p0b.V += aUb[k] * ab[1][k];
    p0b.W += aUb[k] * ab[2][k];
  }
  // V1 = <psi''> U + <c_u psi''>
  R sdum = R(0);
  cmom_psi_b<true, 1, 0, 0>(t0, R(1), V1b, t0b, sdum);
  cmom_psi_b<true, 0, 0, 0>(t0, U, V1b, t0b, p0b.U);
  // tau = 2 mu lam0 / rho0 + tau_add
  const R taub = fit_weights_b(tau, g.dt, g.inv_dt, wFb, wFtb);
  mub += taub * fdiv(R(2) * p0.lam, p0.rho);
  p0b.lam += taub * fdiv(R(2) * g.mu, p0.rho);
  p0b.rho += -taub * fdiv(R(2) * g.mu * p0.lam, p0.rho * p0.rho);
  // slopes abar_i, Abar of g_0
  R ir0b = R(0);
  CSolveB<R> csb;
  csb.e1 = csb.k4 = csb.tlam = R(0);
  centred_slopes_b(p0, ir0, hs2, cs, t0, S.dQ0, abb, Wabb, Abb, Sb.dQ0, ir0b, p0b, hs2b, t0b, csb);
  R hb = R(0);
  centred_solver_b(p0.lam, h, g.K, csb, p0b.lam, hb);
  hb += cent_table_b(h, g.K, t0b);
  p0b.lam += hb * (-h / p0.lam);
  p0b.U += hs2b * U;
  p0b.V += hs2b * V;
  p0b.W += hs2b * W;
  p0b.rho += r0b - ir0b * ir0 * ir0;
  prim_of_b(S.Q0, g.gm1, p0, p0b, Sb.Q0);
}

// VJP of iface_flux: cotangents of (F, F_t) -> of (qL, dqL, qR, dqR) (overwritten) and mu (+=).
// (FTO: zero cotangent of F, Fb not read; the side sums of the heat-flux term,
// which enters F only, are then neither formed nor differentiated)
template <class R, bool FTO = false>
DG_HD void iface_flux_vjp(const R qL[5], const R dqL[3][5], const R qR[5], const R dqR[3][5], const GasPar<R>& g,
                          const R Fb[5], const R Ftb[5], R qLb[5], R dqLb[3][5], R qRb[5], R dqRb[3][5], R& mub) {
  const bool pr_fix = !FTO && (g.pr_fix != R(0));
  SideSums<R> S, Sb;
  iface_zero(S);
  iface_side<R>(1, qL, dqL, g, pr_fix, S);
  iface_side<R>(-1, qR, dqR, g, pr_fix, S);
  iface_finish_b<R, FTO>(S, g, Fb, Ftb, Sb, mub);
  iface_side_b<R>(1, qL, dqL, g, pr_fix, Sb, qLb, dqLb);
  iface_side_b<R>(-1, qR, dqR, g, pr_fix, Sb, qRb, dqRb);
}

// ---- interior flux of one direction ----
// (FTO: zero cotangent of F, Fb not read: only F_t = rho <u_d (A . psi) psi>
// is recomputed and differentiated)
template <int D, bool FTO, class R>
DG_HD void interior_dir_b(const CTab<R>& t, const Prim<R>& p, R hs2, const R a[3][5], const R aU[5], const R A[5],
                          const R Wau[5], R tau, const GasPar<R>& g, const R Fb[5], const R Ftb[5], CTabB<R>& tb,
                          Prim<R>& pb, R& hs2b, R ab[3][5], R aUb[5], R Ab[5], R Waub[5], R& taub) {
  const R Ud = (D == 0) ? p.U : (D == 1) ? p.V : p.W;
  if constexpr (FTO) {
    // F_t = S_U (rho m2), m2 = -Ud Wau + <c_d (A . psi'') psi''>
    R m2[5], Ftc[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) m2[k] = -Ud * Wau[k];
    cmom_a_e<true, D>(t, A, m2);
#pragma unroll
    for (int k = 0; k < 5; ++k) Ftc[k] = p.rho * m2[k];
    R Udb = R(0), Ftcb[5] = {R(0), R(0), R(0), R(0), R(0)}, m2b[5];
    add_uncentred_b<true>(Ftc, p.U, p.V, p.W, hs2, Ftb, Ftcb, pb.U, pb.V, pb.W, hs2b);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      pb.rho += Ftcb[k] * m2[k];
      m2b[k] = Ftcb[k] * p.rho;
      Udb += -m2b[k] * Wau[k];
      Waub[k] += -Ud * m2b[k];
    }
    cmom_a_e_b<true, D>(t, A, m2b, tb, Ab);
    if (D == 0) pb.U += Udb;
    if (D == 1) pb.V += Udb;
    if (D == 2) pb.W += Udb;
    return;
  }
  // forward recomputation (interior_dir)
  R m0[5] = {R(0), R(0), R(0), R(0), R(0)}, m1[5], m2[5];
  cmom_psi<true, 0, 0, 0>(t, Ud, m0);
  cmom_psi<true, D == 0, D == 1, D == 2>(t, R(1), m0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    m1[k] = Ud * Wau[k];
    m2[k] = -Ud * Wau[k];
  }
  cmom_a_ee<true, D, 0>(t, a[0], m1);
  cmom_a_ee<true, D, 1>(t, a[1], m1);
  cmom_a_ee<true, D, 2>(t, a[2], m1);
  cmom_a_e<true, D>(t, aU, m1);
  cmom_a_e<true, D>(t, A, m2);
  R Fc[5], Ftc[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Fc[k] = p.rho * (m0[k] - tau * (m1[k] + m2[k]));
    Ftc[k] = p.rho * m2[k];
  }
  const bool pr_fix = g.pr_fix != R(0);
  R H1 = R(0), H2 = R(0);
  if (pr_fix) {
    H1 = m1[4] - Ud * Wau[4];
    H2 = m2[4] + Ud * Wau[4];
    Fc[4] += g.pr_fix * p.rho * (-tau * (H1 + H2));
  }
  // backward
  R Udb = R(0);
  R Fcb[5] = {R(0), R(0), R(0), R(0), R(0)}, Ftcb[5] = {R(0), R(0), R(0), R(0), R(0)};
  add_uncentred_b<true>(Fc, p.U, p.V, p.W, hs2, Fb, Fcb, pb.U, pb.V, pb.W, hs2b);
  add_uncentred_b<true>(Ftc, p.U, p.V, p.W, hs2, Ftb, Ftcb, pb.U, pb.V, pb.W, hs2b);
  R m0b[5], m1b[5], m2b[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) m0b[k] = m1b[k] = m2b[k] = R(0);
  if (pr_fix) {
    const R H1b = -g.pr_fix * p.rho * tau * Fcb[4];
    const R H2b = -g.pr_fix * p.rho * tau * Fcb[4];
    pb.rho += g.pr_fix * (-tau * (H1 + H2) * Fcb[4]);
    taub += -g.pr_fix * p.rho * (H1 + H2) * Fcb[4];
    m1b[4] += H1b;
    m2b[4] += H2b;
    Udb += (H2b - H1b) * Wau[4];
    Waub[4] += (H2b - H1b) * Ud;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    // Fc = rho (m0 - tau (m1 + m2)), Ftc = rho m2
    pb.rho += Fcb[k] * (m0[k] - tau * (m1[k] + m2[k])) + Ftcb[k] * m2[k];
    taub += -Fcb[k] * p.rho * (m1[k] + m2[k]);
    m0b[k] += Fcb[k] * p.rho;
    m1b[k] += -Fcb[k] * p.rho * tau;
    m2b[k] += -Fcb[k] * p.rho * tau + Ftcb[k] * p.rho;
    // m1 = Ud Wau + ..., m2 = -Ud Wau + ...
    Udb += (m1b[k] - m2b[k]) * Wau[k];
    Waub[k] += Ud * (m1b[k] - m2b[k]);
  }
  cmom_a_e_b<true, D>(t, A, m2b, tb, Ab);
  cmom_a_e_b<true, D>(t, aU, m1b, tb, aUb);
  cmom_a_ee_b<true, D, 2>(t, a[2], m1b, tb, ab[2]);
  cmom_a_ee_b<true, D, 1>(t, a[1], m1b, tb, ab[1]);
  cmom_a_ee_b<true, D, 0>(t, a[0], m1b, tb, ab[0]);
  R sdum = R(0);
  cmom_psi_b<true, D == 0, D == 1, D == 2>(t, R(1), m0b, tb, sdum);
  cmom_psi_b<true, 0, 0, 0>(t, Ud, m0b, tb, Udb);
  if (D == 0) pb.U += Udb;
  if (D == 1) pb.V += Udb;
  if (D == 2) pb.W += Udb;
}

// VJP of interior_flux: cotangents of (F[3][5], F_t[3][5]) -> of (q, dq) (overwritten) and mu (+=).
template <class R, bool FTO = false>
DG_HD void interior_flux_vjp(const R q[5], const R dq[3][5], const GasPar<R>& g, const R Fb[3][5],
                             const R Ftb[3][5], R qb[5], R dqb[3][5], R& mub) {
  // forward recomputation (interior_flux)
  Prim<R> p;
  prim_of(q, g.gm1, p);
  const R ir = fdiv(R(1), p.rho);
  const R h = fdiv(R(0.5), p.lam);
  const R hs2 = R(0.5) * (p.U * p.U + p.V * p.V + p.W * p.W);
  CTab<R> t;
  cent_table(h, g.K, t);
  CSolve<R> cs;
  centred_solver(p.lam, h, g.K, cs);
  R a[3][5], Wau[5], A[5];
  centred_slopes(p, ir, hs2, cs, t, dq, a, Wau, A);
  R aU[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) aU[k] = p.U * a[0][k] + p.V * a[1][k] + p.W * a[2][k];
  const R tau = fdiv(g.mu * R(2) * p.lam, p.rho) + g.tau_add;

  // backward
  CTabB<R> tb;
  ctab_zero(tb);
  Prim<R> pb;
  pb.rho = pb.U = pb.V = pb.W = pb.lam = R(0);
  R hs2b = R(0), taub = R(0);
  R ab[3][5], aUb[5], Ab[5], Waub[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    aUb[k] = Ab[k] = Waub[k] = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) ab[i][k] = R(0);
  }
  interior_dir_b<2, FTO>(t, p, hs2, a, aU, A, Wau, tau, g, Fb[2], Ftb[2], tb, pb, hs2b, ab, aUb, Ab, Waub, taub);
  interior_dir_b<1, FTO>(t, p, hs2, a, aU, A, Wau, tau, g, Fb[1], Ftb[1], tb, pb, hs2b, ab, aUb, Ab, Waub, taub);
  interior_dir_b<0, FTO>(t, p, hs2, a, aU, A, Wau, tau, g, Fb[0], Ftb[0], tb, pb, hs2b, ab, aUb, Ab, Waub, taub);
  // tau = 2 mu lam / rho + tau_add
  mub += taub * fdiv(R(2) * p.lam, p.rho);
  pb.lam += taub * fdiv(R(2) * g.mu, p.rho);
  pb.rho += -taub * fdiv(R(2) * g.mu * p.lam, p.rho * p.rho);
  // aU = U a_0 + V a_1 + W a_2
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    ab[0][k] += p.U * aUb[k];
    ab[1][k] += p.V * aUb[k];
    ab[2][k] += p.W * aUb[k];
    pb.U += aUb[k] * a[0][k];
    pb.V += aUb[k] * a[1][k];
    pb.W += aUb[k] * a[2][k];
  }
  R irb = R(0);
  CSolveB<R> csb;
  csb.e1 = csb.k4 = csb.tlam = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 5; ++k) dqb[i][k] = R(0);
  centred_slopes_b(p, ir, hs2, cs, t, dq, ab, Waub, Ab, dqb, irb, pb, hs2b, tb, csb);
  R hb = R(0);
  centred_solver_b(p.lam, h, g.K, csb, pb.lam, hb);
  hb += cent_table_b(h, g.K, tb);
  pb.lam += hb * (-h / p.lam);
  pb.U += hs2b * p.U;
  pb.V += hs2b * p.V;
  pb.W += hs2b * p.W;
  pb.rho += -irb * ir * ir;
#pragma unroll
  for (int k = 0; k < 5; ++k) qb[k] = R(0);
  prim_of_b(q, g.gm1, p, pb, qb);
}

}  // namespace dghgks

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
//   * Pr != 1 (not in the paper): the energy flux F (not F_t) gains
//     (1/Pr - 1) q, where q = 1/2 <(u_n - U_n)(|u - U|^2 + xi^2) f> is
//     evaluated from the flux moments F = <u_n psi phi> and density moments
//     W = <psi phi> of each term phi of f.  The correction is fitted at t_n
//     only: q is taken about the velocity U of t_n, and the part of f that
//     grows linearly in t moves its mean velocity, so the fitted time
//     derivative of q would carry a frame-shift term proportional to d_t U
//     (not a heat flux); with it the P2 scheme grew its high modes without
//     bound at Pr = 0.72.
//
// Implementation choices (B300): moment indices are template parameters so
// every moment product is resolved at compile time; the 5x5 slope systems are
// solved in closed form; side-local data is folded into running sums
// (Q_0, dQ_0/dn, and the free-transport flux moments) before the other side
// is touched, so the live register set stays small.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <utility>

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
// IEEE operations; the FP32 path uses the approximate PTX instructions of the
// special-function unit with denormal inputs and results flushed to zero
// (about 2 ulp; the exponential as 2^(x log2 e), whose error grows with |x|
// as the product is rounded), which is well inside the FP32-mixed error
// budget and avoids the multi-instruction IEEE sequences and the extra
// instructions that the denormal-preserving forms need.
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
  float r;
  asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float frsqrt<float>(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <>
__device__ __forceinline__ float fexp<float>(float x) {
  // e^x = 2^(x log2 e)
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * 1.4426950408889634f));
  return r;
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
// Moments in a frame that moves with the Maxwellian.
//
// With c = u - s for a shift s, psi = S_s psi' where psi' = (1, c_u, c_v,
// c_w, (|c|^2 + xi^2)/2) and
//   S_s m' = (m'0, m'1 + s_u m'0, m'2 + s_v m'0, m'3 + s_w m'0,
//             m'4 + s . m'_{1..3} + |s|^2/2 m'0),
// so a . psi = (S_s^T a) . psi' and <phi psi> = S_s <phi psi'>; S_a S_b =
// S_{a+b}.  The tangential components are always centred on the Maxwellian's
// velocity (s_v = V, s_w = W); the normal one is centred too (s_u = U, full
// space, CU = true) or not (s_u = 0, the half-space moments of one side of an
// interface, CU = false).  Central moments of odd order of a full-space
// Gaussian vanish, so every moment product containing one is dropped at
// compile time: the 5 x 5 moment matrices <c^ABC psi' psi'^T> keep 11, 6 or
// 2 of their 25 entries.  The results are those of the lab-frame formulas;
// only the rounding order differs.
// ---------------------------------------------------------------------------
template <class R>
struct CTab {
  R u[7];        // <c_u^n>: the raw half-space moments (CU = false)
  R c2, c4, c6;  // central moments of a full-space component: h, 3 h^2, 15 h^3
  R xi2, xi4;    // <xi^2>, <xi^4>
};

template <class R>
DG_HD void cent_table(R h, R K, CTab<R>& t) {
  t.c2 = h;
  t.c4 = R(3) * h * h;
  t.c6 = R(15) * h * h * h;
  t.xi2 = K * h;
  t.xi4 = K * (K + R(2)) * h * h;
}

template <bool CU, int A, int B, int C>
constexpr bool cm_zero() {
  return (B % 2) || (C % 2) || (CU && (A % 2));
}
template <int N, class R>
DG_HD R cm_c(const CTab<R>& t) {  // central moment of even order N of a full-space component
  static_assert(N % 2 == 0 && N <= 6, "central moment out of table");
  if constexpr (N == 0) return R(1);
  else if constexpr (N == 2) return t.c2;
  else if constexpr (N == 4) return t.c4;
  else return t.c6;
}
// <c_u^A c_v^B c_w^C>, for a non-vanishing moment only
template <bool CU, int A, int B, int C, class R>
DG_HD R cm(const CTab<R>& t) {
  static_assert(!cm_zero<CU, A, B, C>(), "vanishing moment");
  static_assert(A <= 6, "moment power out of table");
  R x;
  if constexpr (CU) x = cm_c<A>(t);
  else x = t.u[A];
  if constexpr (B > 0) x = x * cm_c<B>(t);
  if constexpr (C > 0) x = x * cm_c<C>(t);
  return x;
}
// <c^ABC psi'_4> and <c^ABC psi'_4^2> (same parity as <c^ABC>)
template <bool CU, int A, int B, int C, class R>
DG_HD R cm5(const CTab<R>& t) {
  return R(0.5) * (cm<CU, A + 2, B, C>(t) + cm<CU, A, B + 2, C>(t) + cm<CU, A, B, C + 2>(t) + t.xi2 * cm<CU, A, B, C>(t));
}
template <bool CU, int A, int B, int C, class R>
DG_HD R cm55(const CTab<R>& t) {
  return R(0.25) * (cm<CU, A + 4, B, C>(t) + cm<CU, A, B + 4, C>(t) + cm<CU, A, B, C + 4>(t) +
                    R(2) * (cm<CU, A + 2, B + 2, C>(t) + cm<CU, A + 2, B, C + 2>(t) + cm<CU, A, B + 2, C + 2>(t)) +
                    R(2) * t.xi2 * (cm<CU, A + 2, B, C>(t) + cm<CU, A, B + 2, C>(t) + cm<CU, A, B, C + 2>(t)) +
                    t.xi4 * cm<CU, A, B, C>(t));
}
// <c^ABC psi'_J psi'_K> (psi'_0 = 1, psi'_{1,2,3} = c_{u,v,w}, psi'_4 even)
template <bool CU, int J, int K, int A, int B, int C>
constexpr bool ent_zero() {
  return cm_zero<CU, A + (J == 1) + (K == 1), B + (J == 2) + (K == 2), C + (J == 3) + (K == 3)>();
}
template <bool CU, int J, int K, int A, int B, int C, class R>
DG_HD R ent(const CTab<R>& t) {
  if constexpr (J == 4 && K == 4) return cm55<CU, A, B, C>(t);
  else if constexpr (J == 4) return cm5<CU, A + (K == 1), B + (K == 2), C + (K == 3)>(t);
  else if constexpr (K == 4) return cm5<CU, A + (J == 1), B + (J == 2), C + (J == 3)>(t);
  else return cm<CU, A + (J == 1) + (K == 1), B + (J == 2) + (K == 2), C + (J == 3) + (K == 3)>(t);
}

template <bool CU, int A, int B, int C, int K, int J, class R>
DG_HD void cmom_a_term(const CTab<R>& t, const R a[5], R out[5]) {
  if constexpr (!ent_zero<CU, J, K, A, B, C>()) out[K] += a[J] * ent<CU, J, K, A, B, C>(t);
}
template <bool CU, int A, int B, int C, class R, int... I>
DG_HD void cmom_a_seq(const CTab<R>& t, const R a[5], R out[5], std::integer_sequence<int, I...>) {
  (cmom_a_term<CU, A, B, C, I / 5, I % 5>(t, a, out), ...);
}
// out += <c^ABC (a . psi') psi'>
template <bool CU, int A, int B, int C, class R>
DG_HD void cmom_a(const CTab<R>& t, const R a[5], R out[5]) {
  cmom_a_seq<CU, A, B, C>(t, a, out, std::make_integer_sequence<int, 25>{});
}
// out += s <c^ABC psi'>
template <bool CU, int A, int B, int C, class R>
DG_HD void cmom_psi(const CTab<R>& t, R s, R out[5]) {
  if constexpr (!ent_zero<CU, 0, 0, A, B, C>()) out[0] += s * ent<CU, 0, 0, A, B, C>(t);
  if constexpr (!ent_zero<CU, 0, 1, A, B, C>()) out[1] += s * ent<CU, 0, 1, A, B, C>(t);
  if constexpr (!ent_zero<CU, 0, 2, A, B, C>()) out[2] += s * ent<CU, 0, 2, A, B, C>(t);
  if constexpr (!ent_zero<CU, 0, 3, A, B, C>()) out[3] += s * ent<CU, 0, 3, A, B, C>(t);
  if constexpr (!ent_zero<CU, 0, 4, A, B, C>()) out[4] += s * ent<CU, 0, 4, A, B, C>(t);
}
// out += <c_D (a . psi') psi'>, D = 0, 1, 2 (u, v, w)
template <bool CU, int D, class R>
DG_HD void cmom_a_e(const CTab<R>& t, const R a[5], R out[5]) {
  cmom_a<CU, D == 0, D == 1, D == 2>(t, a, out);
}
// out += <c_D c_E (a . psi') psi'>
template <bool CU, int D, int E, class R>
DG_HD void cmom_a_ee(const CTab<R>& t, const R a[5], R out[5]) {
  cmom_a<CU, (D == 0) + (E == 0), (D == 1) + (E == 1), (D == 2) + (E == 2)>(t, a, out);
}

// m'' = S_{-s} m (lab -> frame centred on s = (U, V, W)); hs2 = |s|^2 / 2
template <class R>
DG_HD void to_centred(const R m[5], R U, R V, R W, R hs2, R out[5]) {
  out[0] = m[0];
  out[1] = m[1] - U * m[0];
  out[2] = m[2] - V * m[0];
  out[3] = m[3] - W * m[0];
  out[4] = m[4] - U * m[1] - V * m[2] - W * m[3] + hs2 * m[0];
}
// out += S_s m' (frame centred on s -> lab); SU = false for s_u = 0
template <bool SU, class R>
DG_HD void add_uncentred(const R mp[5], R U, R V, R W, R hs2, R out[5]) {
  out[0] += mp[0];
  if constexpr (SU) {
    out[1] += mp[1] + U * mp[0];
    out[4] += mp[4] + U * mp[1] + V * mp[2] + W * mp[3] + hs2 * mp[0];
  } else {
    out[1] += mp[1];
    out[4] += mp[4] + V * mp[2] + W * mp[3] + hs2 * mp[0];
  }
  out[2] += mp[2] + V * mp[0];
  out[3] += mp[3] + W * mp[0];
}

// Closed-form solution of <(a . psi'') psi''> = b for the full-space
// Maxwellian in its own frame: the moment matrix has <1> = 1, <c_i^2> = h,
// <psi''_4> = (K+3) h / 2 = e1 and <psi''_4^2> - e1^2 = (K+3) h^2 / 2, so
// a_i = b_i / h, a_4 = (b_4 - e1 b_0) 2 / ((K+3) h^2), a_0 = b_0 - e1 a_4.
template <class R>
struct CSolve {
  R e1;    // <psi''_4>
  R k4;    // 2 / ((K+3) h^2) = 8 lam^2 / (K+3)
  R tlam;  // 1 / h = 2 lam
};
template <class R>
DG_HD void centred_solver(R lam, R h, R K, CSolve<R>& cs) {
  cs.e1 = R(0.5) * (K + R(3)) * h;
  cs.k4 = fdiv(R(8) * lam * lam, K + R(3));
  cs.tlam = R(2) * lam;
}
template <class R>
DG_HD void centred_solve(const CSolve<R>& cs, const R b[5], R a[5]) {
  a[4] = cs.k4 * (b[4] - cs.e1 * b[0]);
  a[1] = cs.tlam * b[1];
  a[2] = cs.tlam * b[2];
  a[3] = cs.tlam * b[3];
  a[0] = b[0] - cs.e1 * a[4];
}

// Coefficients in the frame centred on s -> in the frame centred on s + (d, 0, 0)
// (c_u = c_u' + d): a' = S_{(d,0,0)}^T a, in place
template <class R>
DG_HD void coef_shift_u(R a[5], R d) {
  a[0] = a[0] + d * a[1] + R(0.5) * d * d * a[4];
  a[1] = a[1] + d * a[4];
}

// Slopes of one state in its own frame: a''_i from the derivatives dq_i
// (b_i = dq_i / rho taken to the centred frame), the centred right-hand sides
// b''_i, and the compatibility condition <A psi> = -<(a . u) psi> for A'',
// whose right-hand side -Wau'' is returned too (u_i = c_i + U_i, and
// <(a''_i . psi'') psi''> = b''_i).
template <class R>
DG_HD void centred_slopes(const Prim<R>& p, R ir, R hs2, const CSolve<R>& cs, const CTab<R>& t, const R dq[3][5],
                          R a[3][5], R Wau[5], R A[5]) {
  const R Uc[3] = {p.U, p.V, p.W};
#pragma unroll
  for (int k = 0; k < 5; ++k) Wau[k] = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R b[5], bc[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k] = dq[i][k] * ir;
    to_centred(b, p.U, p.V, p.W, hs2, bc);
    centred_solve(cs, bc, a[i]);
#pragma unroll
    for (int k = 0; k < 5; ++k) Wau[k] += Uc[i] * bc[k];
  }
  cmom_a_e<true, 0>(t, a[0], Wau);
  cmom_a_e<true, 1>(t, a[1], Wau);
  cmom_a_e<true, 2>(t, a[2], Wau);
  R bA[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) bA[k] = -Wau[k];
  centred_solve(cs, bA, A);
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
// value so that a kernel can loop over the two sides without unrolling.  The
// slopes are solved in the state's own frame; the half-space moments are
// taken in the frame centred on (0, V, W) and added to the sums in the lab
// (local) frame.
template <class R>
DG_HD bool iface_side(int SGN, const R q[5], const R dq[3][5], const GasPar<R>& g, bool pr_fix,
                      SideSums<R>& S) {
  Prim<R> p;
  const bool ok = prim_of(q, g.gm1, p);
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
  // to the frame centred on (0, V, W), scaled by rho (the moments are linear in them)
  const R r = p.rho;
  coef_shift_u(A, -p.U);
#pragma unroll
  for (int k = 0; k < 5; ++k) A[k] = r * A[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    coef_shift_u(a[i], -p.U);
#pragma unroll
    for (int k = 0; k < 5; ++k) a[i][k] = r * a[i][k];
  }
  // sum_i u_i a_i with u_2 = c_v + V, u_3 = c_w + W: the shifted parts
  R aVW[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) aVW[k] = p.V * a[1][k] + p.W * a[2][k];
  // half-space table along the normal
  half_line(t.u, p.U, p.lam, h, SGN);
  // each sum: its moments in the frame of the table, then added in the lab frame
  R m[5] = {R(0), R(0), R(0), R(0), R(0)};
  auto add_to = [&](R dst[5]) {
    add_uncentred<false>(m, R(0), p.V, p.W, ht2, dst);
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k] = R(0);
  };
  cmom_psi<false, 0, 0, 0>(t, r, m);
  add_to(S.Q0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cmom_a<false, 0, 0, 0>(t, a[i], m);
    add_to(S.dQ0[i]);
  }
  cmom_psi<false, 1, 0, 0>(t, r, m);
  add_to(S.V4);
  cmom_a<false, 2, 0, 0>(t, a[0], m);
  cmom_a<false, 1, 1, 0>(t, a[1], m);
  cmom_a<false, 1, 0, 1>(t, a[2], m);
  cmom_a<false, 1, 0, 0>(t, aVW, m);
  add_to(S.V5);
  cmom_a<false, 1, 0, 0>(t, A, m);
  add_to(S.V6);
  if (pr_fix) {
    cmom_a<false, 1, 0, 0>(t, a[0], m);
    cmom_a<false, 0, 1, 0>(t, a[1], m);
    cmom_a<false, 0, 0, 1>(t, a[2], m);
    cmom_a<false, 0, 0, 0>(t, aVW, m);
    add_to(S.W5);
    cmom_a<false, 0, 0, 0>(t, A, m);
    add_to(S.W6);
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
// the flux (local frame) from the side sums of both sides; the g_0 terms are
// formed in the frame of g_0.
template <class R>
DG_HD bool iface_finish(const SideSums<R>& S, const GasPar<R>& g, R F[5], R Ft[5]) {
  const bool pr_fix = (g.pr_fix != R(0));
  Prim<R> p0;
  const bool ok = prim_of(S.Q0, g.gm1, p0);
  const R ir0 = fdiv(R(1), p0.rho);
  const R h = fdiv(R(0.5), p0.lam);
  const R U = p0.U, V = p0.V, W = p0.W;
  const R hs2 = R(0.5) * (U * U + V * V + W * W);
  CTab<R> t0;
  cent_table(h, g.K, t0);
  CSolve<R> cs;
  centred_solver(p0.lam, h, g.K, cs);
  R ab[3][5], Wab[5], Ab[5];  // abar_i, <(abar . u) psi>, Abar (frame of g_0)
  centred_slopes(p0, ir0, hs2, cs, t0, S.dQ0, ab, Wab, Ab);

  // collision time and fit weights
  const R tau = fdiv(g.mu * R(2) * p0.lam, p0.rho) + g.tau_add;  // mu / p_0 + tau_eps dt
  R wF[6], wFt[6];
  fit_weights(tau, g.dt, g.inv_dt, wF, wFt);

  // g_0 terms (per unit density): V1 = <u psi>, V2 = <u (abar . u) psi>,
  // V3 = <u Abar psi>, with u = c_u + U, u_i = c_i + U_i
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
  // free-transport sums in the frame of g_0
  R V4[5], V5[5], V6[5];
  to_centred(S.V4, U, V, W, hs2, V4);
  to_centred(S.V5, U, V, W, hs2, V5);
  to_centred(S.V6, U, V, W, hs2, V6);
  const R r0 = p0.rho;
  R Fc[5], Ftc[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Fc[k] = r0 * (wF[0] * V1[k] + wF[1] * V2[k] + wF[2] * V3[k]) + wF[3] * V4[k] + wF[4] * V5[k] + wF[5] * V6[k];
    Ftc[k] = r0 * (wFt[0] * V1[k] + wFt[1] * V2[k] + wFt[2] * V3[k]) + wFt[3] * V4[k] + wFt[4] * V5[k] +
             wFt[5] * V6[k];
  }
  if (pr_fix) {
    // heat moments 1/2 <c_u (|c|^2 + xi^2) phi> = <c_u psi''_4 phi> of terms 2..6 (term 1, g_0
    // itself, carries none): component 4 of <u psi'' phi> - U <psi'' phi>
    auto c4 = [&](const R m[5]) { return m[4] - U * m[1] - V * m[2] - W * m[3] + hs2 * m[0]; };
    const R H2 = r0 * (V2[4] - U * Wab[4]);
    const R H3 = r0 * (V3[4] + U * Wab[4]);
    const R H4 = V4[4] - U * c4(S.Q0);
    const R H5 = V5[4] - U * c4(S.W5);
    const R H6 = V6[4] - U * c4(S.W6);
    Fc[4] += g.pr_fix * (wF[1] * H2 + wF[2] * H3 + wF[3] * H4 + wF[4] * H5 + wF[5] * H6);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = Ft[k] = R(0);
  add_uncentred<true>(Fc, U, V, W, hs2, F);
  add_uncentred<true>(Ftc, U, V, W, hs2, Ft);
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
// Interior flux of Eq. (flux-2) in the global frame: F[d][k], Ft[d][k], formed
// in the frame of the cell-point Maxwellian:
//   m0 = <u_d psi>, m1 = sum_i <u_d u_i (a_i . psi) psi>, m2 = <u_d (A . psi) psi>,
//   F = rho (m0 - tau (m1 + m2)), F_t = rho m2.
// ---------------------------------------------------------------------------
template <int D, class R>
DG_HD void interior_dir(const CTab<R>& t, const Prim<R>& p, R hs2, const R a[3][5], const R aU[5], const R A[5],
                        const R Wau[5], R tau, const GasPar<R>& g, R F[5], R Ft[5]) {
  const R Ud = (D == 0) ? p.U : (D == 1) ? p.V : p.W;
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
  if (g.pr_fix != R(0)) {
    // heat moments about U of the terms (a . u) g and A g: component 4 of
    // <u_d psi'' phi> - U_d <psi'' phi>, with <psi'' (a . u) g> = Wau'' and <psi'' A g> = -Wau''
    // (F only: the t A g term's heat moment about the U of t_n is the frame shift of g)
    const R H1 = m1[4] - Ud * Wau[4];
    const R H2 = m2[4] + Ud * Wau[4];
    Fc[4] += g.pr_fix * p.rho * (-tau * (H1 + H2));
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = Ft[k] = R(0);
  add_uncentred<true>(Fc, p.U, p.V, p.W, hs2, F);
  add_uncentred<true>(Ftc, p.U, p.V, p.W, hs2, Ft);
}

template <class R>
DG_HD bool interior_flux(const R q[5], const R dq[3][5], const GasPar<R>& g, R F[3][5],
                                              R Ft[3][5]) {
  Prim<R> p;
  const bool ok = prim_of(q, g.gm1, p);
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
  interior_dir<0>(t, p, hs2, a, aU, A, Wau, tau, g, F[0], Ft[0]);
  interior_dir<1>(t, p, hs2, a, aU, A, Wau, tau, g, F[1], Ft[1]);
  interior_dir<2>(t, p, hs2, a, aU, A, Wau, tau, g, F[2], Ft[2]);
  return ok;
}

}  // namespace dghgks

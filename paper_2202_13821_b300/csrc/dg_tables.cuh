// Compile-time tables of the modal DG discretisation (Sec. 3 of arXiv:2202.13821).
//
//   * Gauss-Legendre nodes on [-1,1] (ascending) and weights halved so they
//     sum to 1 (the area |Gamma| or volume |K| multiplies them, Eqs. surface
//     and volume).
//   * Legendre polynomials P_0..P_3 and derivatives in closed form.
//   * P_k modes ordered by total degree, pure powers before mixed ones:
//     (000) (100)(010)(001) (200)(020)(002)(110)(101)(011)
//     (300)(030)(003)(210)(201)(120)(021)(102)(012)(111).
//   * Tangential modes of a face (exponents along the two tangential axes,
//     increasing axis order): (00) (10)(01) (20)(02)(11) (30)(03)(21)(12).
#pragma once

namespace dghgks {

__host__ __device__ constexpr double gauss_x(int nq, int a) {
  return nq == 1   ? 0.0
         : nq == 2 ? (a == 0 ? -0.57735026918962576451 : 0.57735026918962576451)
         : nq == 3 ? (a == 0 ? -0.77459666924148337704 : a == 1 ? 0.0 : 0.77459666924148337704)
         : nq == 4 ? (a == 0   ? -0.86113631159405257522
                      : a == 1 ? -0.33998104358485626480
                      : a == 2 ? 0.33998104358485626480
                               : 0.86113631159405257522)
                   : (a == 0   ? -0.90617984593866399280
                      : a == 1 ? -0.53846931010568309104
                      : a == 2 ? 0.0
                      : a == 3 ? 0.53846931010568309104
                               : 0.90617984593866399280);
}

__host__ __device__ constexpr double gauss_w(int nq, int a) {
  return nq == 1   ? 1.0
         : nq == 2 ? 0.5
         : nq == 3 ? (a == 1 ? 0.44444444444444444444 : 0.27777777777777777778)
         : nq == 4 ? ((a == 1 || a == 2) ? 0.32607257743127307131 : 0.17392742256872692869)
                   : (a == 2 ? 0.28444444444444444444 : (a == 1 || a == 3) ? 0.23931433524968323402
                                                                          : 0.11846344252809454376);
}

// Node and weight in the flux precision R, selected in R (no FP64 select or
// conversion in FP32 kernels when the index is a runtime value).
template <class R>
__host__ __device__ __forceinline__ R gauss_xr(int nq, int a) {
  switch (nq) {
    case 1: return R(0.0);
    case 2: return a == 0 ? R(-0.57735026918962576451) : R(0.57735026918962576451);
    case 3: return a == 0 ? R(-0.77459666924148337704) : a == 1 ? R(0.0) : R(0.77459666924148337704);
    case 4:
      return a == 0 ? R(-0.86113631159405257522)
                    : a == 1 ? R(-0.33998104358485626480) : a == 2 ? R(0.33998104358485626480) : R(0.86113631159405257522);
    default:
      return a == 0   ? R(-0.90617984593866399280)
             : a == 1 ? R(-0.53846931010568309104)
             : a == 2 ? R(0.0)
             : a == 3 ? R(0.53846931010568309104)
                      : R(0.90617984593866399280);
  }
}
template <class R>
__host__ __device__ __forceinline__ R gauss_wr(int nq, int a) {
  switch (nq) {
    case 1: return R(1.0);
    case 2: return R(0.5);
    case 3: return a == 1 ? R(0.44444444444444444444) : R(0.27777777777777777778);
    case 4: return (a == 1 || a == 2) ? R(0.32607257743127307131) : R(0.17392742256872692869);
    default:
      return a == 2 ? R(0.28444444444444444444)
                    : (a == 1 || a == 3) ? R(0.23931433524968323402) : R(0.11846344252809454376);
  }
}

template <class R>
__host__ __device__ constexpr R leg(int n, R x) {
  return n == 0 ? R(1) : n == 1 ? x : n == 2 ? R(1.5) * x * x - R(0.5) : R(2.5) * x * x * x - R(1.5) * x;
}
template <class R>
__host__ __device__ constexpr R dleg(int n, R x) {
  return n == 0 ? R(0) : n == 1 ? R(1) : n == 2 ? R(3) * x : R(7.5) * x * x - R(1.5);
}

__host__ __device__ constexpr int n_modes(int order) { return (order + 1) * (order + 2) * (order + 3) / 6; }
__host__ __device__ constexpr int n_tmodes(int order) { return (order + 1) * (order + 2) / 2; }

// exponent of mode m along axis d
__host__ __device__ constexpr int mode_exp(int m, int d) {
  // rows: (nx, ny, nz)
  return (m == 0)    ? 0
         : (m == 1)  ? (d == 0)
         : (m == 2)  ? (d == 1)
         : (m == 3)  ? (d == 2)
         : (m == 4)  ? 2 * (d == 0)
         : (m == 5)  ? 2 * (d == 1)
         : (m == 6)  ? 2 * (d == 2)
         : (m == 7)  ? (d != 2)
         : (m == 8)  ? (d != 1)
         : (m == 9)  ? (d != 0)
         : (m == 10) ? 3 * (d == 0)
         : (m == 11) ? 3 * (d == 1)
         : (m == 12) ? 3 * (d == 2)
         : (m == 13) ? (d == 0 ? 2 : d == 1 ? 1 : 0)
         : (m == 14) ? (d == 0 ? 2 : d == 2 ? 1 : 0)
         : (m == 15) ? (d == 0 ? 1 : d == 1 ? 2 : 0)
         : (m == 16) ? (d == 1 ? 2 : d == 2 ? 1 : 0)
         : (m == 17) ? (d == 0 ? 1 : d == 2 ? 2 : 0)
         : (m == 18) ? (d == 1 ? 1 : d == 2 ? 2 : 0)
                     : 1;  // m == 19: (1,1,1)
}

// tangential mode t -> exponents (p, q)
__host__ __device__ constexpr int tmode_p(int t) {
  return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? 0 : t == 3 ? 2 : t == 4 ? 0 : t == 5 ? 1 : t == 6 ? 3 : t == 7 ? 0 : t == 8 ? 2 : 1;
}
__host__ __device__ constexpr int tmode_q(int t) {
  return t == 0 ? 0 : t == 1 ? 0 : t == 2 ? 1 : t == 3 ? 0 : t == 4 ? 2 : t == 5 ? 1 : t == 6 ? 0 : t == 7 ? 3 : t == 8 ? 1 : 2;
}
__host__ __device__ constexpr int tmode_index(int p, int q) {
  return (p == 0 && q == 0)   ? 0
         : (p == 1 && q == 0) ? 1
         : (p == 0 && q == 1) ? 2
         : (p == 2 && q == 0) ? 3
         : (p == 0 && q == 2) ? 4
         : (p == 1 && q == 1) ? 5
         : (p == 3 && q == 0) ? 6
         : (p == 0 && q == 3) ? 7
         : (p == 2 && q == 1) ? 8
                              : 9;  // (1, 2)
}

// index of the mode of degree <= 2 with exponents (a, b, c) (the inverse of
// mode_exp on the first 10 modes)
__host__ __device__ constexpr int mode_index2(int a, int b, int c) {
  return (a + b + c == 0)         ? 0
         : (a == 1 && b + c == 0) ? 1
         : (b == 1 && a + c == 0) ? 2
         : (c == 1 && a + b == 0) ? 3
         : (a == 2)               ? 4
         : (b == 2)               ? 5
         : (c == 2)               ? 6
         : (a == 1 && b == 1)     ? 7
         : (a == 1 && c == 1)     ? 8
                                  : 9;  // (0, 1, 1)
}

// tangential axes of a face normal to D, in increasing order
__host__ __device__ constexpr int tan1(int D) { return D == 0 ? 1 : 0; }
__host__ __device__ constexpr int tan2(int D) { return D == 2 ? 1 : 2; }

}  // namespace dghgks

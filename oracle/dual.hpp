// Forward-mode dual numbers for the oracle (test infrastructure only).
//
// Dual<double> carries a value and one directional derivative.  Instantiating
// the templated oracle with it gives exact Jacobian-vector products of the
// DG-HGKS residual and step, which the adjoint tests compare against the
// hand-written reverse-mode kernels.  Only elementary rules of calculus are
// used: (fg)' = f'g + fg', (f/g)' = (f'g - fg')/g^2, exp' = exp,
// erfc'(x) = -2/sqrt(pi) exp(-x^2), sqrt'(x) = 1/(2 sqrt(x)).
#pragma once
#include <cmath>

namespace orc {

template <class T>
struct Dual {
  T v{}, d{};
  Dual() = default;
  Dual(double x) : v(x), d(0) {}
  Dual(T x, T dx) : v(x), d(dx) {}
};

template <class T> inline Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <class T> inline Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <class T> inline Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <class T> inline Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> inline Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
template <class T> inline Dual<T> operator+(const Dual<T>& a, double b) { return {a.v + b, a.d}; }
template <class T> inline Dual<T> operator+(double a, const Dual<T>& b) { return {a + b.v, b.d}; }
template <class T> inline Dual<T> operator-(const Dual<T>& a, double b) { return {a.v - b, a.d}; }
template <class T> inline Dual<T> operator-(double a, const Dual<T>& b) { return {a - b.v, -b.d}; }
template <class T> inline Dual<T> operator*(const Dual<T>& a, double b) { return {a.v * b, a.d * b}; }
template <class T> inline Dual<T> operator*(double a, const Dual<T>& b) { return {a * b.v, a * b.d}; }
template <class T> inline Dual<T> operator/(const Dual<T>& a, double b) { return {a.v / b, a.d / b}; }
template <class T> inline Dual<T> operator/(double a, const Dual<T>& b) { return {a / b.v, -a * b.d / (b.v * b.v)}; }
template <class T> inline Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> inline Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }
template <class T> inline Dual<T>& operator*=(Dual<T>& a, const Dual<T>& b) { a = a * b; return a; }
template <class T> inline bool operator<(const Dual<T>& a, const Dual<T>& b) { return a.v < b.v; }
template <class T> inline bool operator>(const Dual<T>& a, const Dual<T>& b) { return a.v > b.v; }
template <class T> inline bool operator<=(const Dual<T>& a, const Dual<T>& b) { return a.v <= b.v; }
template <class T> inline bool operator==(const Dual<T>& a, const Dual<T>& b) { return a.v == b.v; }

template <class T> inline Dual<T> exp(const Dual<T>& a) { T e = std::exp(a.v); return {e, a.d * e}; }
template <class T> inline Dual<T> sqrt(const Dual<T>& a) { T s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
template <class T> inline Dual<T> erfc(const Dual<T>& a) {
  const double two_over_sqrt_pi = 1.12837916709551257390;
  return {std::erfc(a.v), -two_over_sqrt_pi * std::exp(-a.v * a.v) * a.d};
}
template <class T> inline Dual<T> fabs(const Dual<T>& a) { return a.v < 0 ? -a : a; }
template <class T> inline bool isfinite_(const Dual<T>& a) { return std::isfinite(a.v) && std::isfinite(a.d); }
inline bool isfinite_(double a) { return std::isfinite(a); }

inline double value_of(double x) { return x; }
template <class T> inline double value_of(const Dual<T>& x) { return value_of(x.v); }

}  // namespace orc

// Forward-mode dual numbers for the tangent build of the HGKS oracle.
//
// TEST INFRASTRUCTURE ONLY (see hgks_oracle.cpp).  Compiling the oracle with
// -DORACLE_TANGENT makes its scalar type a Dual: every quantity carries its
// value v and its derivative d along one input direction, so one run of the
// unchanged oracle code gives the directional derivative of the step (a
// tangent run).  The value part performs exactly the double operations of the
// plain build, so it reproduces the plain oracle bit for bit.
//
// Derivative rules (calculus, no library code involved):
//   (a +- b)' = a' +- b',  (a b)' = a' b + a b',  (a / b)' = (a' - (a/b) b') / b
//   sqrt(x)' = x' / (2 sqrt(x)),  exp(x)' = exp(x) x'
//   erfc(x)' = -2/sqrt(pi) exp(-x^2) x'
//   |x|' = sign(x) x' with sign(0) = 0 (the convention of the adjoint)
//   (x^e)' = e x^(e-1) x' for a constant exponent e
// Ordering comparisons use the value only.  Equality with a constant asks
// whether the quantity is that constant identically (value AND derivative),
// so that a test "c != 0" skips a term only when it contributes nothing to
// either part.
#pragma once

#include <cmath>

namespace oracle_dual {

struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double x) : v(x), d(0.0) {}  // NOLINT: constants promote implicitly
  Dual(double x, double dx) : v(x), d(dx) {}
  Dual& operator+=(const Dual& b) { d += b.d; v += b.v; return *this; }
  Dual& operator-=(const Dual& b) { d -= b.d; v -= b.v; return *this; }
  Dual& operator*=(const Dual& b) { *this = *this * b; return *this; }
  Dual& operator/=(const Dual& b) { *this = *this / b; return *this; }
  friend Dual operator+(const Dual& a, const Dual& b) { return {a.v + b.v, a.d + b.d}; }
  friend Dual operator-(const Dual& a, const Dual& b) { return {a.v - b.v, a.d - b.d}; }
  friend Dual operator-(const Dual& a) { return {-a.v, -a.d}; }
  friend Dual operator*(const Dual& a, const Dual& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
  friend Dual operator/(const Dual& a, const Dual& b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
  }
  friend bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
  friend bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
  friend bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
  friend bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
  friend bool operator==(const Dual& a, const Dual& b) { return a.v == b.v && a.d == b.d; }
  friend bool operator!=(const Dual& a, const Dual& b) { return !(a == b); }
};

inline Dual sqrt(const Dual& x) {
  const double s = std::sqrt(x.v);
  return {s, x.d / (2.0 * s)};
}
inline Dual exp(const Dual& x) {
  const double e = std::exp(x.v);
  return {e, e * x.d};
}
inline Dual erfc(const Dual& x) {
  const double two_over_sqrt_pi = 1.12837916709551257390;  // 2 / sqrt(pi)
  return {std::erfc(x.v), -two_over_sqrt_pi * std::exp(-x.v * x.v) * x.d};
}
inline Dual fabs(const Dual& x) {
  const double s = x.v > 0.0 ? 1.0 : (x.v < 0.0 ? -1.0 : 0.0);
  return {std::fabs(x.v), s * x.d};
}
inline Dual pow(const Dual& x, double e) {
  const double p = std::pow(x.v, e);
  return {p, e * std::pow(x.v, e - 1.0) * x.d};
}

inline double value(const Dual& x) { return x.v; }
inline double tangent(const Dual& x) { return x.d; }

}  // namespace oracle_dual

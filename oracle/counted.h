// Operation-counting scalar for the counting build of the HGKS oracle.
//
// TEST INFRASTRUCTURE ONLY (see hgks_oracle.cpp).  Compiling the oracle with
// -DORACLE_COUNT (and without OpenMP, so that one thread runs) makes its
// scalar type a Counted: a double that tallies every arithmetic operation it
// takes part in.  The values are exactly those of the plain build; the
// tallies give the oracle's own floating-point work per cell and step:
// additions and subtractions, multiplications, divisions (FP contraction is
// off, so there are no fused operations), and the calls of sqrt, exp, erfc
// and pow, counted separately.  Comparisons and |x| are not counted.
#pragma once

#include <cmath>

namespace oracle_count {

struct Tally {
  unsigned long long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, erfc = 0, pow = 0;
};
inline Tally g_tally;

struct Counted {
  double v = 0.0;
  Counted() = default;
  Counted(double x) : v(x) {}  // NOLINT: constants promote implicitly
  Counted& operator+=(const Counted& b) { ++g_tally.add; v += b.v; return *this; }
  Counted& operator-=(const Counted& b) { ++g_tally.add; v -= b.v; return *this; }
  Counted& operator*=(const Counted& b) { ++g_tally.mul; v *= b.v; return *this; }
  Counted& operator/=(const Counted& b) { ++g_tally.div; v /= b.v; return *this; }
  friend Counted operator+(const Counted& a, const Counted& b) { ++g_tally.add; return {a.v + b.v}; }
  friend Counted operator-(const Counted& a, const Counted& b) { ++g_tally.add; return {a.v - b.v}; }
  friend Counted operator-(const Counted& a) { return {-a.v}; }
  friend Counted operator*(const Counted& a, const Counted& b) { ++g_tally.mul; return {a.v * b.v}; }
  friend Counted operator/(const Counted& a, const Counted& b) { ++g_tally.div; return {a.v / b.v}; }
  friend bool operator<(const Counted& a, const Counted& b) { return a.v < b.v; }
  friend bool operator>(const Counted& a, const Counted& b) { return a.v > b.v; }
  friend bool operator<=(const Counted& a, const Counted& b) { return a.v <= b.v; }
  friend bool operator>=(const Counted& a, const Counted& b) { return a.v >= b.v; }
  friend bool operator==(const Counted& a, const Counted& b) { return a.v == b.v; }
  friend bool operator!=(const Counted& a, const Counted& b) { return a.v != b.v; }
};

inline Counted sqrt(const Counted& x) { ++g_tally.sqrt; return {std::sqrt(x.v)}; }
inline Counted exp(const Counted& x) { ++g_tally.exp; return {std::exp(x.v)}; }
inline Counted erfc(const Counted& x) { ++g_tally.erfc; return {std::erfc(x.v)}; }
inline Counted fabs(const Counted& x) { return {std::fabs(x.v)}; }
inline Counted pow(const Counted& x, double e) { ++g_tally.pow; return {std::pow(x.v, e)}; }

inline double value(const Counted& x) { return x.v; }

}  // namespace oracle_count

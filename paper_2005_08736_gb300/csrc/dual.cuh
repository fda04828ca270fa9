// Forward-mode dual numbers for the adjoint kernels: value and one tangent.
// The device arithmetic of physics.cuh and recon.cuh is templated on its
// number type, so instantiating it with Dual<T> yields exact directional
// derivatives of the same code; the adjoint kernels use them for the
// Jacobians of the point-wise nonlinear maps (interface flux, compatibility
// state, nonlinear WENO weights).
//
// Conventions at non-differentiable points: d|x|/dx = sign(x) with sign(0) = 0.
#pragma once

#include <type_traits>

#include "physics.cuh"

namespace hgks {

template <class T>
struct Dual {
  T v, d;
  __host__ __device__ __forceinline__ Dual() : v(T(0)), d(T(0)) {}
  // A constant: any arithmetic value, zero tangent.
  template <class U, class = typename std::enable_if<std::is_arithmetic<U>::value>::type>
  __host__ __device__ __forceinline__ Dual(U value) : v(T(value)), d(T(0)) {}
  __host__ __device__ __forceinline__ Dual(T value, T tangent) : v(value), d(tangent) {}
};

template <class T> HGKS_HD Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> HGKS_HD Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> HGKS_HD Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> HGKS_HD Dual<T> operator*(Dual<T> a, Dual<T> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <class T> HGKS_HD Dual<T> operator/(Dual<T> a, Dual<T> b) {
  const T inv = T(1) / b.v;
  const T q = a.v * inv;
  return {q, (a.d - q * b.d) * inv};
}
template <class T> HGKS_HD Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a = a + b; return a; }
template <class T> HGKS_HD Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a = a - b; return a; }
template <class T> HGKS_HD Dual<T>& operator*=(Dual<T>& a, Dual<T> b) { a = a * b; return a; }
template <class T> HGKS_HD bool operator<(Dual<T> a, Dual<T> b) { return a.v < b.v; }
template <class T> HGKS_HD bool operator>(Dual<T> a, Dual<T> b) { return a.v > b.v; }

template <class T> HGKS_HD Dual<T> tsqrt(Dual<T> x) {
  const T s = tsqrt(x.v);
  return {s, x.d / (T(2) * s)};
}
template <class T> HGKS_HD Dual<T> texp(Dual<T> x) {
  const T e = texp(x.v);
  return {e, e * x.d};
}
template <class T> HGKS_HD Dual<T> texpm1(Dual<T> x) {
  return {texpm1(x.v), texp(x.v) * x.d};
}
template <class T> HGKS_HD Dual<T> terf(Dual<T> x) {
  // d erf(x)/dx = 2 exp(-x^2) / sqrt(pi)
  return {terf(x.v), T(1.1283791670955126) * texp(-x.v * x.v) * x.d};
}
template <class T> HGKS_HD Dual<T> tpow(Dual<T> x, Dual<T> y) {
  const T p = tpow(x.v, y.v);
  T d = y.v * tpow(x.v, y.v - T(1)) * x.d;
  if (y.d != T(0)) d += p * log(x.v) * y.d;
  return {p, d};
}
template <class T> HGKS_HD Dual<T> tabs(Dual<T> x) {
  const T s = x.v > T(0) ? T(1) : (x.v < T(0) ? T(-1) : T(0));
  return {x.v * s, x.d * s};
}

// Problem constants in dual form (zero tangents).
template <class T>
HGKS_HD Gas<Dual<T>> dual_gas(const Gas<T>& g) {
  Gas<Dual<T>> r;
  r.gamma = g.gamma;
  r.gm1 = g.gm1;
  r.K = g.K;
  r.pr_fix = g.pr_fix;
  r.visc_law = g.visc_law;
  r.mu_ref = g.mu_ref;
  r.T_ref_inv = g.T_ref_inv;
  r.visc_exp = g.visc_exp;
  r.tau_num_C = g.tau_num_C;
  r.rho_r = g.rho_r;
  r.p_r = g.p_r;
  r.h_r = g.h_r;
  return r;
}

}  // namespace hgks

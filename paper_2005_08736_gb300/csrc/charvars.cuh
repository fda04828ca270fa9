// Characteristic variables of the reconstruction (Sec. 2.1, Remark 1):
// omega = R^{-1} Q with R the right eigenvectors of the Jacobian of the
// Euler flux along the face normal (local frame, normal velocity first),
// evaluated at the mean Qm of the two cell averages beside the face point.
//
// Eigenvalues u - c, u, u, u, u + c; columns of R:
//   (1, u - c, v, w, H - u c), (1, u, v, w, |U|^2/2), (0, 0, 1, 0, v),
//   (0, 0, 0, 1, w), (1, u + c, v, w, H + u c),
// H = (rho E + p)/rho, c^2 = gamma p/rho.  Rows of R^{-1}, with
// b1 = (gamma - 1)/c^2 and b2 = b1 |U|^2/2:
//   ((b2 + u/c)/2, -(b1 u + 1/c)/2, -b1 v/2, -b1 w/2, b1/2),
//   (1 - b2, b1 u, b1 v, b1 w, -b1),
//   (-v, 0, 1, 0, 0), (-w, 0, 0, 1, 0),
//   ((b2 - u/c)/2, -(b1 u - 1/c)/2, -b1 v/2, -b1 w/2, b1/2).
// The WENO weights are invariant under adding a constant to a stencil and
// the candidate polynomials are affine, so deviations from the reference
// state (and slopes) are projected directly.
#pragma once

#include "physics.cuh"

namespace hgks {

template <class T>
struct CharBasis {
  T u, v, w, c, ic;  // velocity, sound speed and its reciprocal
  T H, hq2;          // total enthalpy, |U|^2 / 2
  T b1, b2;
};

// Basis at the state Q_ref + dqm.
template <class T>
HGKS_HD CharBasis<T> char_basis(const T dqm[5], const Gas<T>& g) {
  const Prim<T> s = prim_of(dqm, g);
  CharBasis<T> b;
  b.u = s.U;
  b.v = s.V;
  b.w = s.W;
  const T c2 = g.gamma * s.p * s.inv_rho;
  b.c = tsqrt(c2);
  b.ic = T(1) / b.c;
  b.hq2 = T(0.5) * (s.U * s.U + s.V * s.V + s.W * s.W);
  b.H = (g.h_r + dqm[4] + s.dp) * s.inv_rho;
  b.b1 = g.gm1 / c2;
  b.b2 = b.b1 * b.hq2;
  return b;
}

// omega = R^{-1} q
template <class T>
HGKS_HD void to_char(const CharBasis<T>& b, const T q[5], T o[5]) {
  const T k = b.b1 * (b.u * q[1] + b.v * q[2] + b.w * q[3] - q[4]);  // b1 (U.m - E)
  const T a = b.b2 * q[0] - k;                                        // b2 q0 - k
  const T s = (b.u * q[0] - q[1]) * b.ic;                             // (u q0 - q1)/c
  o[0] = T(0.5) * (a + s);
  o[1] = q[0] - a;
  o[2] = q[2] - b.v * q[0];
  o[3] = q[3] - b.w * q[0];
  o[4] = T(0.5) * (a - s);
}

// q = R omega
template <class T>
HGKS_HD void from_char(const CharBasis<T>& b, const T o[5], T q[5]) {
  const T m = o[0] + o[1] + o[4];
  const T d = (o[4] - o[0]) * b.c;
  q[0] = m;
  q[1] = b.u * m + d;
  q[2] = b.v * m + o[2];
  q[3] = b.w * m + o[3];
  q[4] = b.H * (o[0] + o[4]) + b.hq2 * o[1] + b.u * d + b.v * o[2] + b.w * o[3];
}

}  // namespace hgks

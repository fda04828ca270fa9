// Reconstruction of the high-order gas-kinetic scheme (Cao, Pan & Xu,
// arXiv:2005.08736, Sec. 2.1, Remark 1), templated on the floating type T.
//
// Normal direction: fifth-order WENO values at both ends of a cell from the
// cell averages q_{i-2..i+2}; linear weights (smooth flows) or WENO-JS /
// WENO-Z nonlinear weights.  Tangential directions: from five face averages,
// values and derivatives at the two Gauss abscissae s = +-1/(2 sqrt 3) of the
// centre face (cell units) -- the quartic through the five averages for
// linear weights, the quadratic through the WENO end values and the average
// otherwise.
#pragma once

#include "physics.cuh"

namespace hgks {

enum Recon { RECON_LINEAR = 0, RECON_WENO_JS = 1, RECON_WENO_Z = 2 };
enum FluxKind { FLUX_SMOOTH = 0, FLUX_FULL = 1 };

// Kernel template MODE: the Recon value, or Recon + 2 for the WENO modes
// applied to characteristic variables (charvars.cuh): 3 = WENO-JS, 4 = WENO-Z.
// The scalar reconstructions below see the underlying Recon.
template <int MODE> __host__ __device__ constexpr int recon_of() { return MODE >= 3 ? MODE - 2 : MODE; }
template <int MODE> __host__ __device__ constexpr bool is_char_mode() { return MODE >= 3; }

// Both end values of the centre cell: qL at x_{i-1/2}, qR at x_{i+1/2}.
// Candidate quadratics on {i-2,i-1,i}, {i-1,i,i+1}, {i,i+1,i+2} with optimal
// weights (1/10, 6/10, 3/10) for the right end; the left end uses the mirrored
// stencils, whose smoothness indicators are the same three in reverse order.
// WENO-JS: alpha = d/(1e-6 + beta)^2.  WENO-Z: alpha = d (1 + |beta0 - beta2|/(beta + 1e-20)).
template <int MODE_, class T>
HGKS_HD void weno5_pair(T q0, T q1, T q2, T q3, T q4, T& qL, T& qR) {
  constexpr int MODE = recon_of<MODE_>();
  if (MODE == RECON_LINEAR) {
    // The optimal-weight combination of the three candidates is the
    // fifth-degree reconstruction (2, -13, 47, 27, -3)/60 of the five averages.
    const T c60 = T(1) / T(60);
    qR = (T(2) * q0 - T(13) * q1 + T(47) * q2 + T(27) * q3 - T(3) * q4) * c60;
    qL = (T(2) * q4 - T(13) * q3 + T(47) * q2 + T(27) * q1 - T(3) * q0) * c60;
    return;
  }
  const T c6 = T(1) / T(6);
  const T pR0 = (T(2) * q0 - T(7) * q1 + T(11) * q2) * c6;
  const T pR1 = (-q1 + T(5) * q2 + T(2) * q3) * c6;
  const T pR2 = (T(2) * q2 + T(5) * q3 - q4) * c6;
  const T pL0 = (T(2) * q4 - T(7) * q3 + T(11) * q2) * c6;
  const T pL1 = (-q3 + T(5) * q2 + T(2) * q1) * c6;
  const T pL2 = (T(2) * q2 + T(5) * q1 - q0) * c6;
  const T s0 = q0 - T(2) * q1 + q2, t0 = q0 - T(4) * q1 + T(3) * q2;
  const T s1 = q1 - T(2) * q2 + q3, t1 = q1 - q3;
  const T s2 = q2 - T(2) * q3 + q4, t2 = T(3) * q2 - T(4) * q3 + q4;
  const T c13 = T(13) / T(12);
  const T b0 = c13 * s0 * s0 + T(0.25) * t0 * t0;
  const T b1 = c13 * s1 * s1 + T(0.25) * t1 * t1;
  const T b2 = c13 * s2 * s2 + T(0.25) * t2 * t2;
  T f0, f1, f2;  // weight factors of beta0, beta1, beta2
  if (MODE == RECON_WENO_JS) {
    const T e = T(1e-6);
    f0 = T(1) / ((e + b0) * (e + b0));
    f1 = T(1) / ((e + b1) * (e + b1));
    f2 = T(1) / ((e + b2) * (e + b2));
  } else {
    const T e = T(1e-20);
    const T tau5 = tabs(b0 - b2);
    f0 = T(1) + tau5 / (b0 + e);
    f1 = T(1) + tau5 / (b1 + e);
    f2 = T(1) + tau5 / (b2 + e);
  }
  {
    const T a0 = T(0.1) * f0, a1 = T(0.6) * f1, a2 = T(0.3) * f2;
    qR = (a0 * pR0 + a1 * pR1 + a2 * pR2) / (a0 + a1 + a2);
  }
  {
    const T a0 = T(0.1) * f2, a1 = T(0.6) * f1, a2 = T(0.3) * f0;
    qL = (a0 * pL0 + a1 * pL1 + a2 * pL2) / (a0 + a1 + a2);
  }
}

// Tangential reconstruction: values v[m] and derivatives d[m] (per unit of
// cell length) at s_0 = -1/(2 sqrt 3), s_1 = +1/(2 sqrt 3).
// Linear weights: the quartic with the five averages, written as
//   P(+-g)  = E +- O,  E = 719/720 f2 + (f1+f3)/1080 - (f0+f4)/4320,
//                      O = sqrt3 (7/432 (f0-f4) + 25/216 (f3-f1)),
//   P'(+-g) = A +- B,  A = (f0-f4)/12 + 2(f3-f1)/3,
//                      B = sqrt3/54 (-f0 + 13 f1 - 24 f2 + 13 f3 - f4).
// WENO modes: p(s) = a + b s + c s^2 with b = qR - qL, c = 3(qL+qR) - 6 f2,
// a = f2 - c/12, so p(+-g) = f2 +- b g and p'(+-g) = b +- 2 c g.
template <int MODE_, class T>
HGKS_HD void tangential(T f0, T f1, T f2, T f3, T f4, T v[2], T d[2]) {
  constexpr int MODE = recon_of<MODE_>();
  const T sq3 = T(1.7320508075688772);
  if (MODE == RECON_LINEAR) {
    const T E = T(719) / T(720) * f2 + (f1 + f3) * (T(1) / T(1080)) - (f0 + f4) * (T(1) / T(4320));
    const T O = sq3 * (T(7) / T(432) * (f0 - f4) + T(25) / T(216) * (f3 - f1));
    const T A = (f0 - f4) * (T(1) / T(12)) + T(2) / T(3) * (f3 - f1);
    const T B = sq3 / T(54) * (-f0 + T(13) * f1 - T(24) * f2 + T(13) * f3 - f4);
    v[0] = E - O;
    v[1] = E + O;
    d[0] = A - B;
    d[1] = A + B;
  } else {
    T qL, qR;
    weno5_pair<MODE>(f0, f1, f2, f3, f4, qL, qR);
    const T gs = T(0.5) / sq3;
    const T b = qR - qL;
    const T c = T(3) * (qL + qR) - T(6) * f2;
    v[0] = f2 - b * gs;
    v[1] = f2 + b * gs;
    d[0] = b - T(2) * c * gs;
    d[1] = b + T(2) * c * gs;
  }
}

// Values only (for fields whose tangential derivative is not needed).
template <int MODE, class T>
HGKS_HD void tangential_val(T f0, T f1, T f2, T f3, T f4, T v[2]) {
  T d[2];
  tangential<MODE>(f0, f1, f2, f3, f4, v, d);
}

}  // namespace hgks

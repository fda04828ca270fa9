// Device arithmetic of the high-order gas-kinetic scheme (HGKS) of Cao, Pan &
// Xu (arXiv:2005.08736), templated on the floating type T (float or double).
//
// All conservative states handled here are DEVIATIONS from a reference state
// at rest, dQ = Q - Q_ref with Q_ref = (rho_r, 0, 0, 0, p_r/(gamma-1)).  Every
// quantity whose magnitude is set by the reference pressure (pressure,
// enthalpy flux, the Euler momentum flux) is formed from deviations, so that
// FP32 keeps the low-Mach variations instead of rounding them against p_r.
//
// Units: R = 1, p = rho T, lambda = rho / (2 p), theta = 1 / (2 lambda) = T.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

// The arithmetic below is compiled for the device and, where host code
// instantiates it (the operation tally of flopcount.cu), for the host.
#ifndef HGKS_HD
#define HGKS_HD __host__ __device__ __forceinline__
#endif

namespace hgks {

// Problem constants passed by value to every kernel.
template <class T>
struct Gas {
  T gamma, gm1;     // gamma, gamma - 1
  T K;              // internal degrees of freedom N = (5 - 3 gamma)/(gamma - 1), Sec. 2.1
  T pr_fix;         // 1/Pr - 1 (Prandtl fix of the energy flux)
  int visc_law;     // 0 constant, 1 power law
  T mu_ref, T_ref_inv, visc_exp;
  T tau_num_C;      // C of the numerical collision time, Sec. 3 opening
  T rho_r, p_r;     // reference state at rest
  T h_r;            // rho_r E_r + p_r = gamma/(gamma-1) p_r
};

template <class T> HGKS_HD T tsqrt(T x);
template <> HGKS_HD float tsqrt<float>(float x) { return sqrtf(x); }
template <> HGKS_HD double tsqrt<double>(double x) { return sqrt(x); }
template <class T> HGKS_HD T texp(T x);
template <> HGKS_HD float texp<float>(float x) { return expf(x); }
template <> HGKS_HD double texp<double>(double x) { return exp(x); }
template <class T> HGKS_HD T texpm1(T x);
template <> HGKS_HD float texpm1<float>(float x) { return expm1f(x); }
template <> HGKS_HD double texpm1<double>(double x) { return expm1(x); }
template <class T> HGKS_HD T terf(T x);
template <> HGKS_HD float terf<float>(float x) { return erff(x); }
template <> HGKS_HD double terf<double>(double x) { return erf(x); }
template <class T> HGKS_HD T tpow(T x, T y);
template <> HGKS_HD float tpow<float>(float x, float y) { return powf(x, y); }
template <> HGKS_HD double tpow<double>(double x, double y) { return pow(x, y); }
template <class T> HGKS_HD T tabs(T x) { return x < T(0) ? -x : x; }

template <class T>
struct Prim {
  T rho, inv_rho;  // density and its reciprocal
  T U, V, W;       // local-frame velocity
  T dp, p;         // pressure deviation and pressure
  T lam, theta;    // lambda = rho/(2p), theta = 1/(2 lambda)
};

// Primitive variables of the state Q_ref + dq (local frame).
template <class T>
HGKS_HD Prim<T> prim_of(const T dq[5], const Gas<T>& g) {
  Prim<T> s;
  s.rho = g.rho_r + dq[0];
  const T inv = T(1) / s.rho;
  s.inv_rho = inv;
  s.U = dq[1] * inv;
  s.V = dq[2] * inv;
  s.W = dq[3] * inv;
  // p - p_r = (gamma-1) (dE - |m|^2 / (2 rho)); the reference is at rest.
  s.dp = g.gm1 * (dq[4] - T(0.5) * (dq[1] * s.U + dq[2] * s.V + dq[3] * s.W));
  s.p = g.p_r + s.dp;
  s.theta = s.p * inv;
  s.lam = T(0.5) / s.theta;
  return s;
}

// Normalised moments <.> = (1/rho) int g (.) dXi of a Maxwellian.  u may be
// taken over the whole line or over a half line; v, w over the whole line.
template <class T>
struct Mom {
  T u[7], v[7], w[7];
  T xi1, xi2;  // <xi^2> = K theta, <xi^4> = K (K+2) theta^2
};

template <class T>
HGKS_HD void gauss_recursion(T* m, T U, T theta) {
  // <c^(n+2)> = U <c^(n+1)> + (n+1) theta <c^n>, on the line and on half lines.
#pragma unroll
  for (int n = 0; n < 5; ++n) m[n + 2] = U * m[n + 1] + T(n + 1) * theta * m[n];
}

// half: 0 whole line, +1 u > 0, -1 u < 0.
template <class T>
HGKS_HD void moments(const Prim<T>& s, const Gas<T>& g, int half, Mom<T>& m) {
  if (half == 0) {
    m.u[0] = T(1);
    m.u[1] = s.U;
  } else {
    // <u^0>_{u>0} = erfc(-sqrt(lam) U)/2, <u^1>_{u>0} = U <u^0> + exp(-lam U^2)/(2 sqrt(pi lam)).
    const T x = tsqrt(s.lam) * s.U;
    const T e = texp(-x * x) * T(0.28209479177387814) / tsqrt(s.lam);  // 1/(2 sqrt(pi))
    const T sg = T(half);
    m.u[0] = T(0.5) * (T(1) + sg * terf(x));
    m.u[1] = s.U * m.u[0] + sg * e;
  }
  gauss_recursion(m.u, s.U, s.theta);
  m.v[0] = T(1);
  m.v[1] = s.V;
  gauss_recursion(m.v, s.V, s.theta);
  m.w[0] = T(1);
  m.w[1] = s.W;
  gauss_recursion(m.w, s.W, s.theta);
  m.xi1 = g.K * s.theta;
  m.xi2 = g.K * (g.K + T(2)) * s.theta * s.theta;
}

// <u^a v^b w^c>
template <int A, int B, int C, class T>
HGKS_HD T mm(const Mom<T>& m) {
  return m.u[A] * m.v[B] * m.w[C];
}

// <u^a v^b w^c psi>, psi = (1, u, v, w, (u^2+v^2+w^2+xi^2)/2)
template <int A, int B, int C, class T>
HGKS_HD void mom_psi(const Mom<T>& m, T out[5]) {
  const T m0 = mm<A, B, C>(m);
  out[0] = m0;
  out[1] = mm<A + 1, B, C>(m);
  out[2] = mm<A, B + 1, C>(m);
  out[3] = mm<A, B, C + 1>(m);
  out[4] = T(0.5) * (mm<A + 2, B, C>(m) + mm<A, B + 2, C>(m) + mm<A, B, C + 2>(m) + m0 * m.xi1);
}

// <(a.psi) u^a v^b w^c psi>, a.psi = a0 + a1 u + a2 v + a3 w + a4 (u^2+v^2+w^2+xi^2)/2.
template <int A, int B, int C, class T>
HGKS_HD void mom_apsi(const Mom<T>& m, const T a[5], T out[5]) {
  T t0[5], t1[5], t2[5], t3[5], tu[5], tv[5], tw[5];
  mom_psi<A, B, C>(m, t0);
  mom_psi<A + 1, B, C>(m, t1);
  mom_psi<A, B + 1, C>(m, t2);
  mom_psi<A, B, C + 1>(m, t3);
  mom_psi<A + 2, B, C>(m, tu);
  mom_psi<A, B + 2, C>(m, tv);
  mom_psi<A, B, C + 2>(m, tw);
  // <xi^2 u^a v^b w^c psi>: xi^2 multiplies every component, and psi_4 adds xi^4/2.
  const T m0 = mm<A, B, C>(m);
  T tx[5];
  tx[0] = m.xi1 * m0;
  tx[1] = m.xi1 * mm<A + 1, B, C>(m);
  tx[2] = m.xi1 * mm<A, B + 1, C>(m);
  tx[3] = m.xi1 * mm<A, B, C + 1>(m);
  tx[4] = T(0.5) * (m.xi1 * (mm<A + 2, B, C>(m) + mm<A, B + 2, C>(m) + mm<A, B, C + 2>(m)) +
                    m.xi2 * m0);
  const T h = T(0.5) * a[4];
#pragma unroll
  for (int i = 0; i < 5; ++i)
    out[i] = a[0] * t0[i] + a[1] * t1[i] + a[2] * t2[i] + a[3] * t3[i] +
             h * (tu[i] + tv[i] + tw[i] + tx[i]);
}

// Symmetric matrix <u^a v^b w^c psi_i psi_j> (upper triangle, 15 entries in
// the order 00 01 02 03 04 11 12 13 14 22 23 24 33 34 44).
template <int A, int B, int C, class T>
HGKS_HD void mom_psipsi(const Mom<T>& m, T M[15]) {
  const T x1 = m.xi1, x2 = m.xi2;
  const T m0 = mm<A, B, C>(m);
  const T mu1 = mm<A + 1, B, C>(m), mv1 = mm<A, B + 1, C>(m), mw1 = mm<A, B, C + 1>(m);
  const T mu2 = mm<A + 2, B, C>(m), mv2 = mm<A, B + 2, C>(m), mw2 = mm<A, B, C + 2>(m);
  M[0] = m0;
  M[1] = mu1;
  M[2] = mv1;
  M[3] = mw1;
  M[4] = T(0.5) * (mu2 + mv2 + mw2 + m0 * x1);
  M[5] = mu2;
  M[6] = mm<A + 1, B + 1, C>(m);
  M[7] = mm<A + 1, B, C + 1>(m);
  M[8] = T(0.5) * (mm<A + 3, B, C>(m) + mm<A + 1, B + 2, C>(m) + mm<A + 1, B, C + 2>(m) + mu1 * x1);
  M[9] = mv2;
  M[10] = mm<A, B + 1, C + 1>(m);
  M[11] = T(0.5) * (mm<A + 2, B + 1, C>(m) + mm<A, B + 3, C>(m) + mm<A, B + 1, C + 2>(m) + mv1 * x1);
  M[12] = mw2;
  M[13] = T(0.5) * (mm<A + 2, B, C + 1>(m) + mm<A, B + 2, C + 1>(m) + mm<A, B, C + 3>(m) + mw1 * x1);
  M[14] = T(0.25) * (mm<A + 4, B, C>(m) + mm<A, B + 4, C>(m) + mm<A, B, C + 4>(m) +
                     T(2) * (mm<A + 2, B + 2, C>(m) + mm<A + 2, B, C + 2>(m) + mm<A, B + 2, C + 2>(m)) +
                     T(2) * x1 * (mu2 + mv2 + mw2) + x2 * m0);
}

// out += M a for the symmetric matrix M of mom_psipsi.
template <class T>
HGKS_HD void sym5_matvec_add(const T M[15], const T a[5], T out[5]) {
  out[0] += M[0] * a[0] + M[1] * a[1] + M[2] * a[2] + M[3] * a[3] + M[4] * a[4];
  out[1] += M[1] * a[0] + M[5] * a[1] + M[6] * a[2] + M[7] * a[3] + M[8] * a[4];
  out[2] += M[2] * a[0] + M[6] * a[1] + M[9] * a[2] + M[10] * a[3] + M[11] * a[4];
  out[3] += M[3] * a[0] + M[7] * a[1] + M[10] * a[2] + M[12] * a[3] + M[13] * a[4];
  out[4] += M[4] * a[0] + M[8] * a[1] + M[11] * a[2] + M[13] * a[3] + M[14] * a[4];
}

// Solution a of <a.psi psi> = b (moment matrix of the Maxwellian, K internal
// degrees of freedom), in closed form.
template <class T>
HGKS_HD void slope_solve(const Prim<T>& s, const Gas<T>& g, const T b[5],
                                            T a[5]) {
  const T q2 = s.U * s.U + s.V * s.V + s.W * s.W;
  const T k3t = (g.K + T(3)) * s.theta;
  const T l2 = T(2) * s.lam;
  a[4] = (l2 * l2 / (g.K + T(3))) *
         (T(2) * (b[4] - s.U * b[1] - s.V * b[2] - s.W * b[3]) + (q2 - k3t) * b[0]);
  a[3] = l2 * (b[3] - s.W * b[0]) - s.W * a[4];
  a[2] = l2 * (b[2] - s.V * b[0]) - s.V * a[4];
  a[1] = l2 * (b[1] - s.U * b[0]) - s.U * a[4];
  a[0] = b[0] - s.U * a[1] - s.V * a[2] - s.W * a[3] - T(0.5) * a[4] * (q2 + k3t);
}

// <u (a_n.psi u + a_t1.psi v + a_t2.psi w) psi>
template <class T>
HGKS_HD void mom_u_adotu(const Mom<T>& m, const T a[3][5], T out[5]) {
  T r0[5], r1[5], r2[5];
  mom_apsi<2, 0, 0>(m, a[0], r0);
  mom_apsi<1, 1, 0>(m, a[1], r1);
  mom_apsi<1, 0, 1>(m, a[2], r2);
#pragma unroll
  for (int i = 0; i < 5; ++i) out[i] = r0[i] + r1[i] + r2[i];
}

// rho <u psi> - E(Q_ref): the Euler flux of the state minus that of the
// reference state (0, p_r, 0, 0, 0), formed from deviations.
template <class T>
HGKS_HD void euler_flux_dev(const Prim<T>& s, const T dq[5], const Gas<T>& g,
                                               T out[5]) {
  const T m = s.rho * s.U;
  out[0] = m;
  out[1] = m * s.U + s.dp;
  out[2] = m * s.V;
  out[3] = m * s.W;
  out[4] = s.U * (g.h_r + dq[4] + s.dp);
}

// One reconstructed state at a Gauss point: deviation value and derivatives
// along n, t1, t2 (local frame, physical units).
template <class T>
struct PointState {
  T q[5];
  T dq[3][5];
};

// Directional derivative of the Euler flux along local axis J at the state s
// (H = rho E + p) in the direction dQ: J_J(Q) dQ.
template <int J, class T>
HGKS_HD void euler_jvp(const Prim<T>& s, T H, const T dQ[5], const Gas<T>& g,
                                          T out[5]) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
  const T du[3] = {(dQ[1] - U[0] * dQ[0]) * inv, (dQ[2] - U[1] * dQ[0]) * inv,
                   (dQ[3] - U[2] * dQ[0]) * inv};
  const T dp = g.gm1 * (dQ[4] - U[0] * dQ[1] - U[1] * dQ[2] - U[2] * dQ[3] +
                        T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) * dQ[0]);
  const T mJ = s.rho * U[J];
  out[0] = dQ[1 + J];
#pragma unroll
  for (int i = 0; i < 3; ++i) out[1 + i] = dQ[1 + J] * U[i] + mJ * du[i];
  out[1 + J] += dp;
  out[4] = du[J] * H + U[J] * (dQ[4] + dp);
}

// Time derivative of the conservative state of the equilibrium,
// Q_t = rho <A psi> = -rho sum_d <(a_d.psi) u_d psi> = -sum_d J_d(Q) dQ/dx_d:
// each moment of (a.psi) g is the derivative of the Maxwellian's moment along
// the parameter change that a encodes.
template <class T>
HGKS_HD void state_time_derivative(const Prim<T>& s, T H, const T dq[3][5],
                                                      const Gas<T>& g, T Qt[5]) {
  T j0[5], j1[5], j2[5];
  euler_jvp<0>(s, H, dq[0], g, j0);
  euler_jvp<1>(s, H, dq[1], g, j1);
  euler_jvp<2>(s, H, dq[2], g, j2);
#pragma unroll
  for (int i = 0; i < 5; ++i) Qt[i] = -(j0[i] + j1[i] + j2[i]);
}

// Spatial slopes a_n, a_t1, a_t2 from <a_d.psi psi> = (dQ/dx_d)/rho, and the
// time coefficient A from <(a_n u + a_t1 v + a_t2 w + A) psi> = 0 (Sec. 2.1),
// i.e. <A psi> = Q_t / rho.
template <class T>
HGKS_HD void slopes_and_A(const Prim<T>& s, const Gas<T>& g, const T q[5],
                                             const T dq[3][5], T a[3][5], T A[5]) {
  const T inv = s.inv_rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T b[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) b[i] = dq[d][i] * inv;
    slope_solve(s, g, b, a[d]);
  }
  T Qt[5];
  state_time_derivative(s, g.h_r + q[4] + s.dp, dq, g, Qt);
#pragma unroll
  for (int i = 0; i < 5; ++i) Qt[i] *= inv;
  slope_solve(s, g, Qt, A);
}

// Non-equilibrium flux of the smooth BGK solution, -tau rho (<u (a.u) psi> +
// <u A psi>), in its exact closed form: the Navier-Stokes viscous flux of the
// BGK model with mu = tau p, stress mu (grad U + grad U^T) - 2 mu/(K+3) div U I
// (bulk viscosity 2K/(3(K+3)) mu, Sec. 3.1), and heat flux -mu c_p dT/dn
// with c_p = (K+5)/2; `heat_scale` multiplies the heat flux (1/Pr for the
// Prandtl fix).
template <class T>
HGKS_HD void ns_viscous_flux(const Prim<T>& s, const T dq[3][5], const Gas<T>& g,
                                                T mu, T heat_scale, T Fv[5]) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
  // du[j][i] = d u_i / d x_j (local frame) for the entries the normal row needs.
  T du0[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) du0[i] = (dq[0][1 + i] - U[i] * dq[0][0]) * inv;
  const T du10 = (dq[1][1] - U[0] * dq[1][0]) * inv, du11 = (dq[1][2] - U[1] * dq[1][0]) * inv;
  const T du20 = (dq[2][1] - U[0] * dq[2][0]) * inv, du22 = (dq[2][3] - U[2] * dq[2][0]) * inv;
  const T divU = du0[0] + du11 + du22;
  const T q2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const T dp0 = g.gm1 * (dq[0][4] - U[0] * dq[0][1] - U[1] * dq[0][2] - U[2] * dq[0][3] +
                         T(0.5) * q2 * dq[0][0]);
  const T dT0 = (dp0 - s.theta * dq[0][0]) * inv;
  const T s00 = mu * (T(2) * du0[0] - T(2) / (g.K + T(3)) * divU);
  const T s01 = mu * (du0[1] + du10);
  const T s02 = mu * (du0[2] + du20);
  Fv[0] = T(0);
  Fv[1] = -s00;
  Fv[2] = -s01;
  Fv[3] = -s02;
  Fv[4] = -(s00 * U[0] + s01 * U[1] + s02 * U[2]) - heat_scale * mu * T(0.5) * (g.K + T(5)) * dT0;
}

template <class T>
HGKS_HD T viscosity(const Prim<T>& s, const Gas<T>& g) {
  if (g.visc_law == 1) return g.mu_ref * tpow(s.theta * g.T_ref_inv, g.visc_exp);
  return g.mu_ref;
}

// Simplified smooth flux (Sec. 2.1, Remark 1): f = g0 [1 - tau (a.u + A) + t A],
// F = rho0 [<u psi> - tau (<u (a.u) psi> + <u A psi>)], dF = rho0 <u A psi>,
// with tau = mu/p (Sec. 3).  Evaluated through the exact identities
// rho0 <u psi> = Euler flux, -tau rho0 (<u(a.u)psi> + <u A psi>) = BGK
// Navier-Stokes viscous flux, rho0 <u A psi> = J_n(Q0) Q_t.  The Prandtl fix
// scales the heat flux by 1/Pr.  Returns F - E(Q_ref) and dF; want_F = false
// skips F (second S2O4 stage).
template <class T>
HGKS_HD void flux_smooth(const PointState<T>& st0, const Gas<T>& g, bool want_F,
                                            T F[5], T dF[5]) {
  const Prim<T> s = prim_of(st0.q, g);
  const T H = g.h_r + st0.q[4] + s.dp;
  T Qt[5];
  state_time_derivative(s, H, st0.dq, g, Qt);
  euler_jvp<0>(s, H, Qt, g, dF);
  if (!want_F) return;
  T E[5], Fv[5];
  euler_flux_dev(s, st0.q, g, E);
  ns_viscous_flux(s, st0.dq, g, viscosity(s, g), g.pr_fix + T(1), Fv);
#pragma unroll
  for (int i = 0; i < 5; ++i) F[i] = E[i] + Fv[i];
}

// Coefficients of the linear fit F(t) = F + dF t (Eq. (7)) of the six
// time-integrated terms of Eq. (5), in closed form with y = 1 - exp(-dt/(2 tau)),
// r = tau/dt: term k contributes Fq[k] V_k to F and dFq[k] V_k to dF.
template <class T>
HGKS_HD void fit_coefficients(T tau, T dt, T Fq[6], T dFq[6]) {
  const T y = -texpm1(-dt / (T(2) * tau));
  const T eh = T(1) - y;
  const T r = tau / dt;
  const T S = y * (T(2) + y);  // 3 - 4 e^{-dt/2tau} + e^{-dt/tau}
  const T D = y * y;           // (1 - e^{-dt/2tau})^2
  Fq[0] = T(1) - r * S;
  Fq[3] = r * S;
  dFq[0] = T(4) * r * D / dt;
  dFq[3] = -dFq[0];
  Fq[1] = tau * (T(2) * r * S + D - T(2));
  Fq[4] = -tau - Fq[1];
  dFq[1] = T(4) * tau / dt * (eh * y - T(2) * r * D);
  dFq[4] = -dFq[1];
  Fq[2] = -tau * (T(1) - r * S);
  Fq[5] = -tau * r * S;
  dFq[2] = T(1) - T(4) * r * r * D;
  dFq[5] = T(4) * r * r * D;
}

// The full second-order flux (Eq. (5)) in parts, shared by the forward flux
// and its vector-Jacobian product:
//   equilibrium part (state 0): V0 = rho0 <u psi> - E(Q_ref) (Euler flux),
//     V2 = rho0 <u A psi> = J_n Q_t, V1 = rho0 <u (a.u) psi> =
//     -(viscous flux with mu = p, Pr = 1) - V2; mu0, p0 and the normal
//     temperature slope dT0 for tau and the Prandtl fix;
//   half-space part of side l (u > 0, g_l) or r (u < 0, g_r): rho <u psi>,
//     rho <u (a.psi) u_d psi>, rho <u A psi> over the half space, and p;
//   tau = mu0/p0 + C |p_l - p_r|/(p_l + p_r) dt (Sec. 3 opening);
//   the linear fit (Eq. (7)) F = sum_k Fq_k V_k, dF = sum_k dFq_k V_k, and
//   the Prandtl fix of the heat flux.
template <class T>
struct FullEq {
  T V[3][5];
  T mu, p, dT;
};
template <class T>
struct FullSide {
  T V[3][5];
  T p;
};

template <class T>
HGKS_HD void flux_full_eq(const PointState<T>& st0, const Gas<T>& g, FullEq<T>& o) {
  const Prim<T> s = prim_of(st0.q, g);
  const T H = g.h_r + st0.q[4] + s.dp;
  euler_flux_dev(s, st0.q, g, o.V[0]);
  T Qt[5], Fv[5];
  state_time_derivative(s, H, st0.dq, g, Qt);
  euler_jvp<0>(s, H, Qt, g, o.V[2]);
  ns_viscous_flux(s, st0.dq, g, s.p, T(1), Fv);
#pragma unroll
  for (int i = 0; i < 5; ++i) o.V[1][i] = -Fv[i] - o.V[2][i];
  o.mu = viscosity(s, g);
  o.p = s.p;
  // Normal temperature derivative for the Prandtl fix of the heat flux.
  const T q2 = s.U * s.U + s.V * s.V + s.W * s.W;
  const T dp0 = g.gm1 * (st0.dq[0][4] - s.U * st0.dq[0][1] - s.V * st0.dq[0][2] -
                         s.W * st0.dq[0][3] + T(0.5) * q2 * st0.dq[0][0]);
  o.dT = (dp0 - s.theta * st0.dq[0][0]) * s.inv_rho;
}

// side = 0: g_l over u > 0; side = 1: g_r over u < 0.
template <class T>
HGKS_HD void flux_full_side(const PointState<T>& st, const Gas<T>& g, int side,
                                               FullSide<T>& o) {
  const Prim<T> s = prim_of(st.q, g);
  Mom<T> mh;
  T a[3][5], A[5];
  slopes_and_A(s, g, st.q, st.dq, a, A);
  moments(s, g, side == 0 ? +1 : -1, mh);
  // Half-space moments as symmetric matrices: <u psi psi^T>, <u u_d psi psi^T>.
  // <u psi> is the first column of the first; <u (a.psi) u_d psi> = M_d a.
  T ua[5] = {0, 0, 0, 0, 0}, uA[5] = {0, 0, 0, 0, 0};
  T M[15];
  mom_psipsi<1, 0, 0>(mh, M);
#pragma unroll
  for (int i = 0; i < 5; ++i) o.V[0][i] = s.rho * M[i];
  sym5_matvec_add(M, A, uA);
  mom_psipsi<2, 0, 0>(mh, M);
  sym5_matvec_add(M, a[0], ua);
  mom_psipsi<1, 1, 0>(mh, M);
  sym5_matvec_add(M, a[1], ua);
  mom_psipsi<1, 0, 1>(mh, M);
  sym5_matvec_add(M, a[2], ua);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    o.V[1][i] = s.rho * ua[i];
    o.V[2][i] = s.rho * uA[i];
  }
  o.p = s.p;
}

template <class T>
HGKS_HD T collision_time_full(T mu0, T p0, T pl, T pr, const Gas<T>& g, T dt) {
  return mu0 / p0 + g.tau_num_C * tabs((pl - pr) / (pl + pr)) * dt;
}

// The parts of the full flux gathered for one Gauss point: the equilibrium
// part, the sum of the two half-space parts and the pressures of the l and r
// states (the full flux evaluated part by part, state by state).
template <class T>
struct FullParts {
  FullEq<T> e;
  T Vs[3][5];  // half-space parts, side l then + side r
  T pl, pr;
};

// Add the half-space part of side `side` (0: l, assigns; 1: r, adds) of the
// state st to the parts.
template <class T>
HGKS_HD void flux_full_add_side(const PointState<T>& st, const Gas<T>& g, int side, FullParts<T>& a) {
  FullSide<T> h;
  flux_full_side(st, g, side, h);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 5; ++i) a.Vs[k][i] = side == 0 ? h.V[k][i] : a.Vs[k][i] + h.V[k][i];
  if (side == 0) a.pl = h.p; else a.pr = h.p;
}

// The full flux from its parts: tau, the fit of Eq. (7), the Prandtl fix.
template <class T>
HGKS_HD void flux_full_combine(const FullParts<T>& a, const Gas<T>& g, T dt, T F[5], T dF[5]) {
  const FullEq<T>& e = a.e;
  T V[6][5];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      V[k][i] = e.V[k][i];
      V[3 + k][i] = a.Vs[k][i];
    }
  const T pl = a.pl, pr = a.pr;
  V[3][1] -= g.p_r;  // the half-space sum minus the reference Euler flux
  const T tau = collision_time_full(e.mu, e.p, pl, pr, g, dt);
  T Fq[6], dFq[6];
  fit_coefficients(tau, dt, Fq, dFq);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    T f = T(0), df = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      f += Fq[k] * V[k][i];
      df += dFq[k] * V[k][i];
    }
    F[i] = f;
    dF[i] = df;
  }
  // Prandtl fix: (1/Pr - 1) times the heat flux -tau rho0 <h (a.u + A)> =
  // -tau p0 c_p dT/dn of the equilibrium part (tau includes the numerical term).
  F[4] -= g.pr_fix * tau * e.p * (T(0.5) * (g.K + T(5))) * e.dT;
}

// Full second-order flux (Eq. (5)) with the Heaviside factor H(u) on g_l and
// 1 - H(u) on g_r, integrated over [0, dt] and [0, dt/2] and fitted linearly
// (Eq. (7)).  Returns F - E(Q_ref) and dF.
template <class T>
HGKS_HD void flux_full(const PointState<T>& stl, const PointState<T>& str,
                                          const PointState<T>& st0, const Gas<T>& g, T dt,
                                          T F[5], T dF[5]) {
  FullParts<T> a;
  flux_full_eq(st0, g, a.e);
#pragma unroll 1  // one copy of the half-space code for both sides
  for (int side = 0; side < 2; ++side) flux_full_add_side(side == 0 ? stl : str, g, side, a);
  flux_full_combine(a, g, dt, F, dF);
}

// Equilibrium state of the compatibility condition, Q0 = int_{u>0} psi g_l +
// int_{u<0} psi g_r, as a deviation: Q0 - Q_ref = (dQl + dQr)/2 + (S_l - S_r)/2
// with S = int sign(u) psi g = rho (D0, D1, V D0, W D0, (D2 + D0 (V^2+W^2+(K+2) theta))/2),
// D0 = erf(sqrt(lam) U), D1 = U D0 + exp(-lam U^2)/sqrt(pi lam), D2 = U D1 + theta D0.
template <class T>
HGKS_HD void sign_moments(const T dq[5], const Gas<T>& g, T S[5]) {
  const Prim<T> s = prim_of(dq, g);
  const T sl = tsqrt(s.lam);
  const T x = sl * s.U;
  const T D0 = terf(x);
  const T D1 = s.U * D0 + texp(-x * x) * T(0.5641895835477563) * tsqrt(s.theta + s.theta);  // 1/sqrt(pi lam)
  const T D2 = s.U * D1 + s.theta * D0;
  S[0] = s.rho * D0;
  S[1] = s.rho * D1;
  S[2] = s.rho * s.V * D0;
  S[3] = s.rho * s.W * D0;
  S[4] = T(0.5) * s.rho * (D2 + D0 * (s.V * s.V + s.W * s.W + (g.K + T(2)) * s.theta));
}

template <class T>
HGKS_HD void compat_dev(const T dql[5], const T dqr[5], const Gas<T>& g,
                                           T dq0[5]) {
  T Sl[5], Sr[5];
  sign_moments(dql, g, Sl);
  sign_moments(dqr, g, Sr);
#pragma unroll
  for (int i = 0; i < 5; ++i) dq0[i] = T(0.5) * (dql[i] + dqr[i]) + T(0.5) * (Sl[i] - Sr[i]);
}

}  // namespace hgks

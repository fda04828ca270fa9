// Packed FP32 pairs for the sweep kernel: one instruction applies an add,
// multiply or fused multiply-add to both halves of a float2 (__fadd2_rn /
// __fmul2_rn / __ffma2_rn, sm_100 and later).  The sweep kernel is bound by
// instruction issue, not by the FMA pipe, so evaluating two points in the
// halves of one float2 halves the issue slots of their arithmetic.
//
// In the last phase the two halves are the two t1 Gauss abscissae of one
// face; the shared-memory layout of the t1 pass keeps them adjacent, so one
// 64-bit load fetches both.  In the face-field phase they are two adjacent
// points of a face layer (compat.cuh).  The formulas are those of recon.cuh (linear tangential
// reconstruction) and physics.cuh (smooth flux), evaluated pairwise; only the
// rounding of the fused operations can differ from the scalar code.
#pragma once

#include <cmath>

#include "physics.cuh"
#include "recon.cuh"

namespace hgks {

// On the host (the checks of tests/support) each pair operation is the two
// scalar operations it stands for.
HGKS_HD float2 bc2(float s) { return make_float2(s, s); }
HGKS_HD float2 add2(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
HGKS_HD float2 mul2(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
HGKS_HD float2 fma2(float2 a, float2 b, float2 c) {
#if defined(__CUDA_ARCH__)
  return __ffma2_rn(a, b, c);
#else
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
#endif
}
// a - b
HGKS_HD float2 sub2(float2 a, float2 b) { return fma2(b, bc2(-1.f), a); }
HGKS_HD float2 rcp2(float2 a) { return make_float2(1.f / a.x, 1.f / a.y); }

// Linear-weight tangential reconstruction (the quartic through five face
// averages) of two columns at once: values v[m] and derivatives d[m] (per
// unit cell length) at the Gauss abscissae s_m = -+1/(2 sqrt 3):
//   P(+-g) = E +- O,  P'(+-g) = A +- B  with
//   E = 719/720 f2 + (f1+f3)/1080 - (f0+f4)/4320,
//   O = sqrt3 (7/432 (f0-f4) + 25/216 (f3-f1)),
//   A = (f0-f4)/12 + 2(f3-f1)/3,  B = sqrt3/54 (13 (f1+f3) - 24 f2 - (f0+f4)).
HGKS_HD void tangential_linear_x2(float2 f0, float2 f1, float2 f2, float2 f3,
                                                     float2 f4, float2 v[2], float2 d[2]) {
  const float sq3 = 1.7320508075688772f;
  const float2 s13 = add2(f1, f3), s04 = add2(f0, f4);
  const float2 d04 = sub2(f0, f4), d31 = sub2(f3, f1);
  const float2 E = fma2(f2, bc2(719.f / 720.f), fma2(s13, bc2(1.f / 1080.f), mul2(s04, bc2(-1.f / 4320.f))));
  const float2 O = fma2(d04, bc2(sq3 * 7.f / 432.f), mul2(d31, bc2(sq3 * 25.f / 216.f)));
  const float2 A = fma2(d04, bc2(1.f / 12.f), mul2(d31, bc2(2.f / 3.f)));
  const float k = sq3 / 54.f;
  const float2 B = fma2(s13, bc2(13.f * k), fma2(f2, bc2(-24.f * k), mul2(s04, bc2(-k))));
  v[0] = sub2(E, O);
  v[1] = add2(E, O);
  d[0] = sub2(A, B);
  d[1] = add2(A, B);
}

HGKS_HD void tangential_linear_val_x2(float2 f0, float2 f1, float2 f2, float2 f3,
                                                         float2 f4, float2 v[2]) {
  const float sq3 = 1.7320508075688772f;
  const float2 s13 = add2(f1, f3), s04 = add2(f0, f4);
  const float2 d04 = sub2(f0, f4), d31 = sub2(f3, f1);
  const float2 E = fma2(f2, bc2(719.f / 720.f), fma2(s13, bc2(1.f / 1080.f), mul2(s04, bc2(-1.f / 4320.f))));
  const float2 O = fma2(d04, bc2(sq3 * 7.f / 432.f), mul2(d31, bc2(sq3 * 25.f / 216.f)));
  v[0] = sub2(E, O);
  v[1] = add2(E, O);
}

// Two point states (deviation value and derivatives along n, t1, t2, local
// frame), one per half.
struct PointStateX2 {
  float2 q[5];
  float2 dq[3][5];
};

// Velocity gradient and pressure derivative of the state along one axis:
// du[k] = d u_k, dp = d p for the conservative derivative dQ (the pieces the
// Euler Jacobian-vector product and the viscous flux share).
struct DirDeriv {
  float2 du[3], dp;
};

// Smooth BGK flux at two points (physics.cuh, flux_smooth): F - E(Q_ref)
// (want_F) and -dF are accumulated into Fs[0..4] and Fs[5..9] summed over the
// halves: Fs[i] += F_i(.x) + F_i(.y), Fs[5+i] += dF_i(.x) + dF_i(.y).
// dF = J_n(Q0) Q_t with Q_t = -sum_d J_d(Q0) dQ0/dx_d; F = Euler flux + the
// BGK Navier-Stokes viscous flux with the heat flux scaled by 1/Pr.
template <bool WANT_F>
__device__ __forceinline__ void flux_smooth_x2(const PointStateX2& st, const Gas<float>& g, float Fs[10]) {
  // Primitive state (prim_of).
  const float2 rho = add2(bc2(g.rho_r), st.q[0]);
  const float2 inv = rcp2(rho);
  const float2 U[3] = {mul2(st.q[1], inv), mul2(st.q[2], inv), mul2(st.q[3], inv)};
  const float2 nU[3] = {mul2(U[0], bc2(-1.f)), mul2(U[1], bc2(-1.f)), mul2(U[2], bc2(-1.f))};
  const float2 ke2 = fma2(st.q[1], U[0], fma2(st.q[2], U[1], mul2(st.q[3], U[2])));  // |m|^2/rho
  const float2 dp = mul2(bc2(g.gm1), fma2(ke2, bc2(-0.5f), st.q[4]));
  const float2 H = add2(add2(bc2(g.h_r), st.q[4]), dp);
  const float2 hq2 = mul2(bc2(0.5f), fma2(U[0], U[0], fma2(U[1], U[1], mul2(U[2], U[2]))));
  const float2 m[3] = {mul2(rho, U[0]), mul2(rho, U[1]), mul2(rho, U[2])};

  auto deriv = [&](const float2 dQ[5]) {
    DirDeriv r;
#pragma unroll
    for (int k = 0; k < 3; ++k) r.du[k] = mul2(fma2(nU[k], dQ[0], dQ[1 + k]), inv);
    float2 t = fma2(nU[0], dQ[1], dQ[4]);
    t = fma2(nU[1], dQ[2], t);
    t = fma2(nU[2], dQ[3], t);
    t = fma2(hq2, dQ[0], t);
    r.dp = mul2(bc2(g.gm1), t);
    return r;
  };
  // J_J(Q) dQ (euler_jvp) from the shared pieces.
  auto jvp = [&](int J, const float2 dQ[5], const DirDeriv& r, float2 out[5]) {
    out[0] = dQ[1 + J];
#pragma unroll
    for (int i = 0; i < 3; ++i) out[1 + i] = fma2(dQ[1 + J], U[i], mul2(m[J], r.du[i]));
    out[1 + J] = add2(out[1 + J], r.dp);
    out[4] = fma2(r.du[J], H, mul2(U[J], add2(dQ[4], r.dp)));
  };

  const DirDeriv r0 = deriv(st.dq[0]), r1 = deriv(st.dq[1]), r2 = deriv(st.dq[2]);
  // S = sum_d J_d dQ/dx_d = -Q_t.
  float2 S[5], j[5];
  jvp(0, st.dq[0], r0, S);
  jvp(1, st.dq[1], r1, j);
#pragma unroll
  for (int i = 0; i < 5; ++i) S[i] = add2(S[i], j[i]);
  jvp(2, st.dq[2], r2, j);
#pragma unroll
  for (int i = 0; i < 5; ++i) S[i] = add2(S[i], j[i]);
  // dF = J_n Q_t = -J_n S.
  const DirDeriv rs = deriv(S);
  float2 dF[5];
  jvp(0, S, rs, dF);
#pragma unroll
  for (int i = 0; i < 5; ++i) Fs[5 + i] -= dF[i].x + dF[i].y;
  if constexpr (WANT_F) {
    // Viscosity mu(T) of the gas law at T = p/rho.
    float2 mu = bc2(g.mu_ref);
    if (g.visc_law == 1) {
      const float2 th = mul2(add2(bc2(g.p_r), dp), inv);
      mu = make_float2(g.mu_ref * tpow(th.x * g.T_ref_inv, g.visc_exp),
                       g.mu_ref * tpow(th.y * g.T_ref_inv, g.visc_exp));
    }
    // Viscous stress row of the normal direction and the heat flux
    // (ns_viscous_flux) from the gradients of the three directions.
    const float2 theta = mul2(add2(bc2(g.p_r), dp), inv);
    const float2 divU = add2(add2(r0.du[0], r1.du[1]), r2.du[2]);
    const float2 dT0 = mul2(fma2(theta, mul2(st.dq[0][0], bc2(-1.f)), r0.dp), inv);
    const float2 s00 = mul2(mu, fma2(divU, bc2(-2.f / (g.K + 3.f)), mul2(bc2(2.f), r0.du[0])));
    const float2 s01 = mul2(mu, add2(r0.du[1], r1.du[0]));
    const float2 s02 = mul2(mu, add2(r0.du[2], r2.du[0]));
    const float hc = -(g.pr_fix + 1.f) * 0.5f * (g.K + 5.f);
    float2 F[5];
    F[0] = m[0];
    F[1] = sub2(fma2(m[0], U[0], dp), s00);
    F[2] = sub2(mul2(m[0], U[1]), s01);
    F[3] = sub2(mul2(m[0], U[2]), s02);
    const float2 work = fma2(s00, U[0], fma2(s01, U[1], mul2(s02, U[2])));
    F[4] = fma2(mul2(mu, bc2(hc)), dT0, sub2(mul2(U[0], H), work));
#pragma unroll
    for (int i = 0; i < 5; ++i) Fs[i] += F[i].x + F[i].y;
  }
}

// WENO5 end values with nonlinear weights (weno5_pair, WENO-JS or WENO-Z) of
// two columns at once: the candidate polynomials, smoothness indicators,
// weights and combinations in pair arithmetic; |beta0 - beta2| and the
// reciprocals per half.
template <int MODE>
HGKS_HD void weno5_pair_x2(float2 q0, float2 q1, float2 q2, float2 q3, float2 q4,
                                              float2& qL, float2& qR) {
  const float2 c6 = bc2(1.f / 6.f);
  const float2 pR0 = mul2(fma2(bc2(2.f), q0, fma2(bc2(-7.f), q1, mul2(bc2(11.f), q2))), c6);
  const float2 pR1 = mul2(fma2(bc2(-1.f), q1, fma2(bc2(5.f), q2, mul2(bc2(2.f), q3))), c6);
  const float2 pR2 = mul2(fma2(bc2(2.f), q2, fma2(bc2(5.f), q3, mul2(bc2(-1.f), q4))), c6);
  const float2 pL0 = mul2(fma2(bc2(2.f), q4, fma2(bc2(-7.f), q3, mul2(bc2(11.f), q2))), c6);
  const float2 pL1 = mul2(fma2(bc2(-1.f), q3, fma2(bc2(5.f), q2, mul2(bc2(2.f), q1))), c6);
  const float2 pL2 = mul2(fma2(bc2(2.f), q2, fma2(bc2(5.f), q1, mul2(bc2(-1.f), q0))), c6);
  const float2 s0 = fma2(bc2(-2.f), q1, add2(q0, q2)), t0 = fma2(bc2(-4.f), q1, fma2(bc2(3.f), q2, q0));
  const float2 s1 = fma2(bc2(-2.f), q2, add2(q1, q3)), t1 = sub2(q1, q3);
  const float2 s2 = fma2(bc2(-2.f), q3, add2(q2, q4)), t2 = fma2(bc2(3.f), q2, fma2(bc2(-4.f), q3, q4));
  const float2 c13 = bc2(13.f / 12.f), qt = bc2(0.25f);
  const float2 b0 = fma2(mul2(c13, s0), s0, mul2(mul2(qt, t0), t0));
  const float2 b1 = fma2(mul2(c13, s1), s1, mul2(mul2(qt, t1), t1));
  const float2 b2 = fma2(mul2(c13, s2), s2, mul2(mul2(qt, t2), t2));
  float2 f0, f1, f2;  // weight factors of beta0, beta1, beta2
  if constexpr (MODE == RECON_WENO_JS) {
    const float2 e = bc2(1e-6f);
    const float2 e0 = add2(e, b0), e1 = add2(e, b1), e2 = add2(e, b2);
    f0 = rcp2(mul2(e0, e0));
    f1 = rcp2(mul2(e1, e1));
    f2 = rcp2(mul2(e2, e2));
  } else {
    const float2 e = bc2(1e-20f);
    const float2 d02 = sub2(b0, b2);
    const float2 tau5 = make_float2(fabsf(d02.x), fabsf(d02.y));
    f0 = fma2(tau5, rcp2(add2(b0, e)), bc2(1.f));
    f1 = fma2(tau5, rcp2(add2(b1, e)), bc2(1.f));
    f2 = fma2(tau5, rcp2(add2(b2, e)), bc2(1.f));
  }
  {
    const float2 a0 = mul2(bc2(0.1f), f0), a1 = mul2(bc2(0.6f), f1), a2 = mul2(bc2(0.3f), f2);
    qR = mul2(fma2(a0, pR0, fma2(a1, pR1, mul2(a2, pR2))), rcp2(add2(add2(a0, a1), a2)));
  }
  {
    const float2 a0 = mul2(bc2(0.1f), f2), a1 = mul2(bc2(0.6f), f1), a2 = mul2(bc2(0.3f), f0);
    qL = mul2(fma2(a0, pL0, fma2(a1, pL1, mul2(a2, pL2))), rcp2(add2(add2(a0, a1), a2)));
  }
}

// Tangential reconstruction with nonlinear weights (tangential, WENO modes)
// of two columns at once: values v[m] and derivatives d[m] at the two Gauss
// abscissae from the quadratic through the WENO5 end values and the average.
template <int MODE>
HGKS_HD void tangential_weno_x2(float2 f0, float2 f1, float2 f2, float2 f3, float2 f4,
                                                   float2 v[2], float2 d[2]) {
  float2 qL, qR;
  weno5_pair_x2<MODE>(f0, f1, f2, f3, f4, qL, qR);
  const float2 gs = bc2(0.5f / 1.7320508075688772f);
  const float2 b = sub2(qR, qL);
  const float2 c = fma2(bc2(3.f), add2(qL, qR), mul2(bc2(-6.f), f2));
  v[0] = fma2(mul2(b, bc2(-1.f)), gs, f2);
  v[1] = fma2(b, gs, f2);
  const float2 c2 = mul2(mul2(bc2(2.f), c), gs);
  d[0] = sub2(b, c2);
  d[1] = add2(b, c2);
}

}  // namespace hgks

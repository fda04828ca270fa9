// Compatibility state at a face for the sweep kernel: Q0 from the
// compatibility condition of Sec. 2.1 (Eq. (5)), Q0 = int_{u>0} psi g_l +
// int_{u<0} psi g_r, as a deviation from the reference state:
//   Q0 - Q_ref = (dQl + dQr)/2 + (S_l - S_r)/2,
// S = int sign(u) psi g (physics.cuh, sign_moments and compat_dev).
//
// In FP32 the direct difference S_l - S_r loses precision: S carries the
// constant rho sqrt(2 theta / pi) in its momentum component (~7 at Ma 0.1)
// and terms of size p erf(x) in its energy component, while their
// difference is of the size of the jump Ql - Qr, which WENO makes small on
// smooth data.  For small jumps the difference is formed instead by the
// midpoint rule, S_l - S_r = J_S(Q_m) (Ql - Qr) + O(|Ql - Qr|^3), Q_m the
// mean of the two states, the Jacobian-vector product exact (one
// dual-number pass of sign_moments).  Its terms are of the size of the jump,
// so the result keeps FP32's relative precision.  The rule is used when the
// relative jump r = |drho|/rho + |dm|/sqrt(rho p) + (gamma-1)|dE|/p is below
// 2e-3, where the dropped third-order term is below 3e-9 of |S| (~2e-8
// absolute in the energy at Ma 0.1, under the FP32 rounding of Q0); larger
// jumps take the direct difference, whose cancellation is then mild.  FP64
// always takes the direct difference.
#pragma once

#include <type_traits>

#include "dual.cuh"
#include "packed.cuh"

namespace hgks {

// Whether the midpoint rule applies to the jump dd about the mean dm (FP32).
__device__ __forceinline__ bool compat_small_jump(const float dm[5], const float dd[5], const Gas<float>& g) {
  const float rho = g.rho_r + dm[0];
  const float ke2 = (dm[1] * dm[1] + dm[2] * dm[2] + dm[3] * dm[3]) / rho;
  const float p = g.p_r + g.gm1 * (dm[4] - 0.5f * ke2);
  const float r = fabsf(dd[0]) / rho + (fabsf(dd[1]) + fabsf(dd[2]) + fabsf(dd[3])) * rsqrtf(rho * p) +
                  g.gm1 * fabsf(dd[4]) / p;
  return r < 2e-3f && rho > 0.f && p > 0.f;
}

template <class T>
HGKS_HD void compat_state(const T dql[5], const T dqr[5], const Gas<T>& g, T dq0[5]) {
  if constexpr (std::is_same<T, float>::value) {
    float dm[5], dd[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      dm[i] = 0.5f * (dql[i] + dqr[i]);
      dd[i] = dql[i] - dqr[i];
    }
    if (compat_small_jump(dm, dd, g)) {
      Dual<float> q[5], S[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) q[i] = Dual<float>(dm[i], dd[i]);
      sign_moments(q, dual_gas(g), S);
#pragma unroll
      for (int i = 0; i < 5; ++i) dq0[i] = dm[i] + 0.5f * S[i].d;
      return;
    }
  }
  compat_dev(dql, dqr, g, dq0);
}

// Midpoint-rule jump of the sign moments for two points at once (packed
// pairs, packed.cuh helpers): 0.5 J_S(Q_m)(Ql - Qr) from the means dm and
// jumps dd of two faces, the tangent of sign_moments written out by the
// chain rule (prime = derivative along dd):
//   rho' = dd0, inv' = -inv rho' inv, U_k' = (dd_k - U_k rho') inv,
//   dp' = gm1 (dd4 - (U.dd_m) + |U|^2 rho'/2), theta' = (dp' - theta rho') inv,
//   lam = 1/(2 theta), sl = sqrt(lam), sl' = -sl theta'/(2 theta),
//   x = sl U, x' = sl' U + sl U', D0' = 2/sqrt(pi) e x' (e = exp(-x^2)),
//   R = sqrt(2 theta), R' = theta'/R, D1 = U D0 + e R/sqrt(pi) ... c = 1/sqrt(pi),
//   D1' = U' D0 + U D0' + c (R' - 2 x x' R) e,
//   D2 = U D1 + theta D0, D2' = U' D1 + U D1' + theta' D0 + theta D0',
//   S0' = rho' D0 + rho D0', S1' = rho' D1 + rho D1',
//   S2' = dd2 D0 + m2 D0', S3' = dd3 D0 + m3 D0',
//   S4 = rho (D2 + D0 G)/2 with G = V^2 + W^2 + (K+2) theta:
//   S4' = (rho' (D2 + D0 G) + rho (D2' + D0' G + D0 G'))/2,
//   G' = 2 V V' + 2 W W' + (K+2) theta'.
// Returns 0.5 S' per component (the caller adds the mean dm).
__device__ __forceinline__ void compat_jump_x2(const float2 dm[5], const float2 dd[5], const Gas<float>& g,
                                               float2 half_dS[5]) {
  const float2 rho = add2(bc2(g.rho_r), dm[0]);
  const float2 inv = rcp2(rho);
  const float2 U = mul2(dm[1], inv), V = mul2(dm[2], inv), W = mul2(dm[3], inv);
  const float2 rp = dd[0];
  const float2 Up = mul2(fma2(mul2(U, bc2(-1.f)), rp, dd[1]), inv);
  const float2 Vp = mul2(fma2(mul2(V, bc2(-1.f)), rp, dd[2]), inv);
  const float2 Wp = mul2(fma2(mul2(W, bc2(-1.f)), rp, dd[3]), inv);
  const float2 q2 = fma2(U, U, fma2(V, V, mul2(W, W)));
  const float2 ke2 = fma2(dm[1], U, fma2(dm[2], V, mul2(dm[3], W)));
  const float2 dp = mul2(bc2(g.gm1), fma2(ke2, bc2(-0.5f), dm[4]));
  const float2 theta = mul2(add2(bc2(g.p_r), dp), inv);
  // dp' = gm1 (dd4 - U.dd_m + |U|^2 rho'/2)
  const float2 udm = fma2(U, dd[1], fma2(V, dd[2], mul2(W, dd[3])));
  const float2 dpp = mul2(bc2(g.gm1), fma2(mul2(q2, bc2(0.5f)), rp, sub2(dd[4], udm)));
  const float2 thp = mul2(fma2(mul2(theta, bc2(-1.f)), rp, dpp), inv);
  const float2 tt = add2(theta, theta);
  const float2 R = make_float2(sqrtf(tt.x), sqrtf(tt.y));   // sqrt(2 theta)
  const float2 sl = rcp2(R);                                 // sqrt(lambda) = 1/sqrt(2 theta)
  const float2 slp = mul2(mul2(sl, bc2(-0.5f)), mul2(thp, rcp2(theta)));
  const float2 x = mul2(sl, U);
  const float2 xp = fma2(slp, U, mul2(sl, Up));
  const float2 D0 = make_float2(erff(x.x), erff(x.y));
  const float2 e = make_float2(expf(-x.x * x.x), expf(-x.y * x.y));
  const float c = 0.5641895835477563f;  // 1/sqrt(pi)
  const float2 D0p = mul2(bc2(2.f * c), mul2(e, xp));
  const float2 Rp = mul2(thp, sl);
  const float2 D1 = fma2(U, D0, mul2(bc2(c), mul2(e, R)));
  // (R' - 2 x x' R) e
  const float2 er = mul2(e, fma2(mul2(bc2(-2.f), mul2(x, xp)), R, Rp));
  const float2 D1p = fma2(Up, D0, fma2(U, D0p, mul2(bc2(c), er)));
  const float2 D2 = fma2(U, D1, mul2(theta, D0));
  const float2 D2p = fma2(Up, D1, fma2(U, D1p, fma2(thp, D0, mul2(theta, D0p))));
  const float2 G = fma2(V, V, fma2(W, W, mul2(bc2(g.K + 2.f), theta)));
  const float2 Gp = fma2(mul2(bc2(2.f), V), Vp, fma2(mul2(bc2(2.f), W), Wp, mul2(bc2(g.K + 2.f), thp)));
  half_dS[0] = mul2(bc2(0.5f), fma2(rp, D0, mul2(rho, D0p)));
  half_dS[1] = mul2(bc2(0.5f), fma2(rp, D1, mul2(rho, D1p)));
  half_dS[2] = mul2(bc2(0.5f), fma2(dd[2], D0, mul2(dm[2], D0p)));
  half_dS[3] = mul2(bc2(0.5f), fma2(dd[3], D0, mul2(dm[3], D0p)));
  const float2 inner = fma2(D0, G, D2);
  const float2 innerp = fma2(D0p, G, fma2(D0, Gp, D2p));
  half_dS[4] = mul2(bc2(0.25f), fma2(rp, inner, mul2(rho, innerp)));
}

// Face fields of the smooth flux (Q0 and its normal slope) at two adjacent
// points of a face layer: qk[i][k] = variable i of cell f-3+k at both points
// (conservative variables, linear weights; face_fields_cells in sweep.cuh).
// The WENO5 end values and the normal slope in pair arithmetic, the
// compatibility state per point (compat.cuh).
__device__ __forceinline__ void face_fields_smooth_linear_x2(const float2 qk[5][6], float hl, float hr,
                                                             const Gas<float>& g, float2 Q0[5],
                                                             float2 D0[5]) {
  const float r6 = 1.f / (6.f * (hl + hr));
  const float c60 = 1.f / 60.f;
  float2 Ql[5], Qr[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float2* q = qk[i];
    // WENO5 end values with the optimal weights: (2, -13, 47, 27, -3)/60.
    float2 t = mul2(bc2(2.f), q[0]);
    t = fma2(bc2(-13.f), q[1], t);
    t = fma2(bc2(47.f), q[2], t);
    t = fma2(bc2(27.f), q[3], t);
    t = fma2(bc2(-3.f), q[4], t);
    Ql[i] = mul2(t, bc2(c60));
    float2 u = mul2(bc2(2.f), q[5]);
    u = fma2(bc2(-13.f), q[4], u);
    u = fma2(bc2(47.f), q[3], u);
    u = fma2(bc2(27.f), q[2], u);
    u = fma2(bc2(-3.f), q[1], u);
    Qr[i] = mul2(u, bc2(c60));
    float2 w = sub2(q[1], mul2(bc2(15.f), q[2]));
    w = fma2(bc2(15.f), q[3], w);
    D0[i] = mul2(sub2(w, q[4]), bc2(r6));
  }
  // The compatibility state (compat.cuh): the midpoint rule in pair
  // arithmetic when both points' jumps are small, else per point.
  float2 dm[5], dd[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    dm[i] = mul2(bc2(0.5f), add2(Ql[i], Qr[i]));
    dd[i] = sub2(Ql[i], Qr[i]);
  }
  bool small = true;
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    float m[5], j[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      m[i] = hh ? dm[i].y : dm[i].x;
      j[i] = hh ? dd[i].y : dd[i].x;
    }
    small = small && compat_small_jump(m, j, g);
  }
  if (small) {
    float2 half_dS[5];
    compat_jump_x2(dm, dd, g, half_dS);
#pragma unroll
    for (int i = 0; i < 5; ++i) Q0[i] = add2(dm[i], half_dS[i]);
    return;
  }
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    float ql[5], qr[5], q0[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      ql[i] = hh ? Ql[i].y : Ql[i].x;
      qr[i] = hh ? Qr[i].y : Qr[i].x;
    }
    compat_state(ql, qr, g, q0);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (hh) Q0[i].y = q0[i];
      else Q0[i].x = q0[i];
    }
  }
}

}  // namespace hgks

// Adjoint (vector-Jacobian product) of one stage evaluation of the HGKS
// operator: given cotangents w_L, w_dL of L(Q) and dL(Q)/dt on the cells,
// accumulate sum_c (w_L . dL_c/dQ + w_dL . d(dL_c)/dQ) into a padded cotangent
// buffer.  There is no counterpart in the paper (its scheme has no adjoint);
// the step's adjoint is assembled from two such evaluations in hgks_api.cu.
//
// The kernel mirrors the forward sweep (sweep.cuh) tile by tile and layer by
// layer.  For each face layer it first recomputes the face fields and the t1
// pass into shared memory, then runs the reverse:
//   R3  per Gauss point: the cotangent of the face flux from the divergence
//       (Eq. (4)), the vector-Jacobian product of the flux at the point, and
//       the transposed t2 pass, accumulated into shared memory;
//   R2  the transposed t1 pass into face-field cotangents;
//   R1  per transverse point: the compatibility state, the normal slopes and
//       the WENO5 pairs transposed, scattered into the cells f-3 .. f+2 with
//       atomics.
// The WENO5 end values and the tangential polynomials are transposed in
// reverse mode (closed-form derivatives of the nonlinear weights); the flux's
// slope inputs through the transposes of the linear maps that consume them;
// the flux's values in reverse mode through each part of the flux
// (flux_rev.cuh), and the compatibility state's sign moments likewise.
// Ghost cells collect cotangents like interior cells; k_fold_ghosts returns
// them to their periodic images afterwards.
#pragma once

#include "dual.cuh"
#include "flux_rev.cuh"
#include "packed.cuh"
#include "sweep.cuh"

namespace hgks {

// cot[j] += gL dqL/dq_j + gR dqR/dq_j for the WENO5 end values of the centre
// cell (weno5_pair), in reverse mode: q_end = sum_k a_k p_k / sum_k a_k, so
// the cotangent of p_k is g a_k/S and that of a_k is g (p_k - q_end)/S; the
// weights' factors f_k depend on the smoothness indicators beta_k (WENO-JS:
// f = (eps + beta)^-2; WENO-Z: f = 1 + tau5/(beta + eps), tau5 = |beta0 -
// beta2|, d|x|/dx = sign(x) with sign(0) = 0), each a quadratic form of q.
template <int MODE_, class T>
HGKS_HD void weno5_pair_vjp(const T q[5], T gL, T gR, T cot[5]) {
  constexpr int MODE = recon_of<MODE_>();
  const T c6 = T(1) / T(6);
  // Candidate polynomials: d pR_k / dq and d pL_k / dq (times 6).
  const T dR[3][5] = {{2, -7, 11, 0, 0}, {0, -1, 5, 2, 0}, {0, 0, 2, 5, -1}};
  const T dL[3][5] = {{0, 0, 11, -7, 2}, {0, 2, 5, -1, 0}, {-1, 5, 2, 0, 0}};
  if constexpr (MODE == RECON_LINEAR) {
    const T w[3] = {T(0.1), T(0.6), T(0.3)};
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cot[j] += (gR * w[k] * dR[k][j] + gL * w[k] * dL[k][j]) * c6;
  } else {
    T pR[3], pL[3];
  #pragma unroll
    for (int k = 0; k < 3; ++k) {
      pR[k] = T(0);
      pL[k] = T(0);
  #pragma unroll
      for (int j = 0; j < 5; ++j) {
        pR[k] += dR[k][j] * q[j];
        pL[k] += dL[k][j] * q[j];
      }
      pR[k] *= c6;
      pL[k] *= c6;
    }
    const T sv[3] = {q[0] - T(2) * q[1] + q[2], q[1] - T(2) * q[2] + q[3], q[2] - T(2) * q[3] + q[4]};
    const T tv[3] = {q[0] - T(4) * q[1] + T(3) * q[2], q[1] - q[3], T(3) * q[2] - T(4) * q[3] + q[4]};
    const T c13 = T(13) / T(12);
    T bt[3], f[3];
  #pragma unroll
    for (int k = 0; k < 3; ++k) bt[k] = c13 * sv[k] * sv[k] + T(0.25) * tv[k] * tv[k];
    T tau5 = T(0), sg = T(0);
    if (MODE == RECON_WENO_JS) {
  #pragma unroll
      for (int k = 0; k < 3; ++k) f[k] = T(1) / ((T(1e-6) + bt[k]) * (T(1e-6) + bt[k]));
    } else {
      const T d02 = bt[0] - bt[2];
      tau5 = tabs(d02);
      sg = d02 > T(0) ? T(1) : (d02 < T(0) ? T(-1) : T(0));
  #pragma unroll
      for (int k = 0; k < 3; ++k) f[k] = T(1) + tau5 / (bt[k] + T(1e-20));
    }
    const T aR[3] = {T(0.1) * f[0], T(0.6) * f[1], T(0.3) * f[2]};
    const T aL[3] = {T(0.1) * f[2], T(0.6) * f[1], T(0.3) * f[0]};
    const T iSR = T(1) / (aR[0] + aR[1] + aR[2]), iSL = T(1) / (aL[0] + aL[1] + aL[2]);
    const T qR = (aR[0] * pR[0] + aR[1] * pR[1] + aR[2] * pR[2]) * iSR;
    const T qL = (aL[0] * pL[0] + aL[1] * pL[1] + aL[2] * pL[2]) * iSL;
    T gaR[3], gaL[3];
  #pragma unroll
    for (int k = 0; k < 3; ++k) {
      gaR[k] = gR * (pR[k] - qR) * iSR;
      gaL[k] = gL * (pL[k] - qL) * iSL;
    }
    const T gf[3] = {T(0.1) * gaR[0] + T(0.3) * gaL[2], T(0.6) * (gaR[1] + gaL[1]),
                     T(0.3) * gaR[2] + T(0.1) * gaL[0]};
    T gb[3];
    if (MODE == RECON_WENO_JS) {
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T e = T(1e-6) + bt[k];
        gb[k] = gf[k] * T(-2) / (e * e * e);
      }
    } else {
      T gtau = T(0);
  #pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T ie = T(1) / (bt[k] + T(1e-20));
        gb[k] = -gf[k] * tau5 * ie * ie;
        gtau += gf[k] * ie;
      }
      gb[0] += gtau * sg;
      gb[2] -= gtau * sg;
    }
    // beta_k = 13/12 s_k^2 + t_k^2 / 4, s_k and t_k linear in q.
    const T ds[3][5] = {{1, -2, 1, 0, 0}, {0, 1, -2, 1, 0}, {0, 0, 1, -2, 1}};
    const T dt[3][5] = {{1, -4, 3, 0, 0}, {0, 1, 0, -1, 0}, {0, 0, 3, -4, 1}};
  #pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T gs = gb[k] * T(2) * c13 * sv[k], gt = gb[k] * T(0.5) * tv[k];
      const T gpR = gR * aR[k] * iSR * c6, gpL = gL * aL[k] * iSL * c6;
  #pragma unroll
      for (int j = 0; j < 5; ++j) cot[j] += gs * ds[k][j] + gt * dt[k][j] + gpR * dR[k][j] + gpL * dL[k][j];
    }
  }
}

// weno5_pair_vjp (nonlinear weights) for two stencils at once, in the
// halves of packed FP32 pairs: the forward quantities and the reverse pass
// of the scalar function, pairwise; |beta0 - beta2|, its sign and the
// reciprocals per half.
template <int MODE>
HGKS_HD void weno5_pair_vjp_x2(const float2 q[5], float2 gL, float2 gR, float2 cot[5]) {
  const float c6 = 1.f / 6.f;
  const float dR[3][5] = {{2, -7, 11, 0, 0}, {0, -1, 5, 2, 0}, {0, 0, 2, 5, -1}};
  const float dL[3][5] = {{0, 0, 11, -7, 2}, {0, 2, 5, -1, 0}, {-1, 5, 2, 0, 0}};
  float2 pR[3], pL[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pR[k] = bc2(0.f);
    pL[k] = bc2(0.f);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      if (dR[k][j] != 0.f) pR[k] = fma2(bc2(dR[k][j]), q[j], pR[k]);
      if (dL[k][j] != 0.f) pL[k] = fma2(bc2(dL[k][j]), q[j], pL[k]);
    }
    pR[k] = mul2(pR[k], bc2(c6));
    pL[k] = mul2(pL[k], bc2(c6));
  }
  const float2 sv[3] = {fma2(bc2(-2.f), q[1], add2(q[0], q[2])), fma2(bc2(-2.f), q[2], add2(q[1], q[3])),
                        fma2(bc2(-2.f), q[3], add2(q[2], q[4]))};
  const float2 tv[3] = {fma2(bc2(-4.f), q[1], fma2(bc2(3.f), q[2], q[0])), sub2(q[1], q[3]),
                        fma2(bc2(3.f), q[2], fma2(bc2(-4.f), q[3], q[4]))};
  const float c13 = 13.f / 12.f;
  float2 bt[3], f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) bt[k] = fma2(mul2(bc2(c13), sv[k]), sv[k], mul2(mul2(bc2(0.25f), tv[k]), tv[k]));
  float2 tau5 = bc2(0.f), sg = bc2(0.f);
  if constexpr (MODE == RECON_WENO_JS) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 e = add2(bc2(1e-6f), bt[k]);
      f[k] = rcp2(mul2(e, e));
    }
  } else {
    const float2 d02 = sub2(bt[0], bt[2]);
    tau5 = make_float2(fabsf(d02.x), fabsf(d02.y));
    sg = make_float2(d02.x > 0.f ? 1.f : (d02.x < 0.f ? -1.f : 0.f), d02.y > 0.f ? 1.f : (d02.y < 0.f ? -1.f : 0.f));
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = fma2(tau5, rcp2(add2(bt[k], bc2(1e-20f))), bc2(1.f));
  }
  const float2 aR[3] = {mul2(bc2(0.1f), f[0]), mul2(bc2(0.6f), f[1]), mul2(bc2(0.3f), f[2])};
  const float2 aL[3] = {mul2(bc2(0.1f), f[2]), mul2(bc2(0.6f), f[1]), mul2(bc2(0.3f), f[0])};
  const float2 iSR = rcp2(add2(add2(aR[0], aR[1]), aR[2])), iSL = rcp2(add2(add2(aL[0], aL[1]), aL[2]));
  const float2 qR = mul2(fma2(aR[0], pR[0], fma2(aR[1], pR[1], mul2(aR[2], pR[2]))), iSR);
  const float2 qL = mul2(fma2(aL[0], pL[0], fma2(aL[1], pL[1], mul2(aL[2], pL[2]))), iSL);
  float2 gaR[3], gaL[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gaR[k] = mul2(mul2(gR, sub2(pR[k], qR)), iSR);
    gaL[k] = mul2(mul2(gL, sub2(pL[k], qL)), iSL);
  }
  const float2 gf[3] = {fma2(bc2(0.1f), gaR[0], mul2(bc2(0.3f), gaL[2])), mul2(bc2(0.6f), add2(gaR[1], gaL[1])),
                        fma2(bc2(0.3f), gaR[2], mul2(bc2(0.1f), gaL[0]))};
  float2 gb[3];
  if constexpr (MODE == RECON_WENO_JS) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 e = add2(bc2(1e-6f), bt[k]);
      gb[k] = mul2(mul2(gf[k], bc2(-2.f)), rcp2(mul2(mul2(e, e), e)));
    }
  } else {
    float2 gtau = bc2(0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // (-gf tau5 ie) ie, in the scalar order: ie^2 alone overflows FP32
      // where beta vanishes (ie = 1e20), and tau5 = 0 there.
      const float2 ie = rcp2(add2(bt[k], bc2(1e-20f)));
      gb[k] = mul2(mul2(mul2(mul2(gf[k], bc2(-1.f)), tau5), ie), ie);
      gtau = fma2(gf[k], ie, gtau);
    }
    gb[0] = fma2(gtau, sg, gb[0]);
    gb[2] = fma2(mul2(gtau, bc2(-1.f)), sg, gb[2]);
  }
  // beta_k = 13/12 s_k^2 + t_k^2 / 4, s_k and t_k linear in q.
  const float ds[3][5] = {{1, -2, 1, 0, 0}, {0, 1, -2, 1, 0}, {0, 0, 1, -2, 1}};
  const float dt[3][5] = {{1, -4, 3, 0, 0}, {0, 1, 0, -1, 0}, {0, 0, 3, -4, 1}};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 gs = mul2(gb[k], mul2(bc2(2.f * c13), sv[k])), gt = mul2(gb[k], mul2(bc2(0.5f), tv[k]));
    const float2 gpR = mul2(mul2(gR, aR[k]), mul2(iSR, bc2(c6))), gpL = mul2(mul2(gL, aL[k]), mul2(iSL, bc2(c6)));
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      if (ds[k][j] != 0.f) cot[j] = fma2(gs, bc2(ds[k][j]), cot[j]);
      if (dt[k][j] != 0.f) cot[j] = fma2(gt, bc2(dt[k][j]), cot[j]);
      if (dR[k][j] != 0.f) cot[j] = fma2(gpR, bc2(dR[k][j]), cot[j]);
      if (dL[k][j] != 0.f) cot[j] = fma2(gpL, bc2(dL[k][j]), cot[j]);
    }
  }
}

// tangential_vjp (nonlinear weights) of two five-point stencils at once.
template <int MODE>
HGKS_HD void tangential_vjp_x2(const float2 f[5], const float2 gv[2], const float2 gd[2],
                                                  float2 cot[5]) {
  const float gs = 0.5f / 1.7320508075688772f;
  const float2 gb = fma2(bc2(gs), sub2(gv[1], gv[0]), add2(gd[0], gd[1]));
  const float2 gc = mul2(bc2(2.f * gs), sub2(gd[1], gd[0]));
  cot[2] = add2(cot[2], fma2(bc2(-6.f), gc, add2(gv[0], gv[1])));
  weno5_pair_vjp_x2<MODE>(f, fma2(bc2(3.f), gc, mul2(gb, bc2(-1.f))), fma2(bc2(3.f), gc, gb), cot);
}

// cot[j] += sum_m gv[m] dv[m]/df_j + gd[m] dd[m]/df_j for the tangential
// polynomial of the five averages f (the transpose of tangential()).
template <int MODE_, class T>
HGKS_HD void tangential_vjp(const T f[5], const T gv[2], const T gd[2],
                                               T cot[5]) {
  constexpr int MODE = recon_of<MODE_>();
  const T sq3 = T(1.7320508075688772);
  if (MODE == RECON_LINEAR) {
    // v = E -+ O, d = A -+ B (quartic through the five averages)
    const T gE = gv[0] + gv[1], gO = gv[1] - gv[0], gA = gd[0] + gd[1], gB = gd[1] - gd[0];
    const T e0 = T(1) / T(4320), e1 = T(1) / T(1080), e2 = T(719) / T(720);
    const T o0 = sq3 * T(7) / T(432), o1 = sq3 * T(25) / T(216);
    const T a0 = T(1) / T(12), a1 = T(2) / T(3);
    const T b0 = sq3 / T(54);
    cot[0] += -gE * e0 + gO * o0 + gA * a0 - gB * b0;
    cot[1] += gE * e1 - gO * o1 - gA * a1 + gB * b0 * T(13);
    cot[2] += gE * e2 - gB * b0 * T(24);
    cot[3] += gE * e1 + gO * o1 + gA * a1 + gB * b0 * T(13);
    cot[4] += -gE * e0 - gO * o0 - gA * a0 - gB * b0;
    return;
  }
  // p(+-g) = f2 +- b g, p'(+-g) = b +- 2 c g, b = qR - qL, c = 3(qL + qR) - 6 f2.
  const T gs = T(0.5) / sq3;
  const T gb = gs * (gv[1] - gv[0]) + gd[0] + gd[1];
  const T gc = T(2) * gs * (gd[1] - gd[0]);
  cot[2] += gv[0] + gv[1] - T(6) * gc;
  weno5_pair_vjp<MODE>(f, -gb + T(3) * gc, gb + T(3) * gc, cot);
}

// (cl, cr) += J^T g0 for the compatibility state Q0(Q_l, Q_r) =
// (Q_l + Q_r)/2 + (S(Q_l) - S(Q_r))/2 (compat_dev): the identity part
// directly, S of each state by one reverse-mode pass (flux_rev.cuh).
template <class T>
__device__ __forceinline__ void compat_vjp(const T ql[5], const T qr[5], const T g0[5],
                                           const Gas<T>& gas, T cl[5], T cr[5]) {
  T hp[5], hm[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    cl[i] += T(0.5) * g0[i];
    cr[i] += T(0.5) * g0[i];
    hp[i] = T(0.5) * g0[i];
    hm[i] = -T(0.5) * g0[i];
  }
  sign_moments_rev(ql, gas, hp, cl);
  sign_moments_rev(qr, gas, hm, cr);
}

// Cotangents of the reconstructed Gauss-point states (value and the three
// derivatives of each of NS states) from the flux cotangents (gF, gdF).
template <class T, int FLUX>
__device__ __forceinline__ void flux_vjp(const PointState<T>* st, const Gas<T>& gas, T dt,
                                         bool want_F, const T gF[5], const T gdF[5],
                                         PointState<T>* cot) {
  if constexpr (FLUX == FLUX_FULL) flux_full_vjp(st, gas, dt, gF, gdF, cot);
  else flux_smooth_rev(st[0], gas, want_F, gF, gdF, cot[0]);
}

template <class T>
struct AdjArgs {
  const T* __restrict__ q;      // padded state (deviation) with ghost cells filled
  const T* __restrict__ wL;     // cotangent of L, [5][N] (null: zero)
  const T* __restrict__ wdL;    // cotangent of dL/dt, [5][N]
  T* __restrict__ acc;          // padded cotangent of the state, [5][P], accumulated
  const T* __restrict__ wn;
  const T* __restrict__ wt1;
  const T* __restrict__ wt2;
  const double* __restrict__ scal;
  GridDev g;
  int d;
  int chunk;
  Gas<T> gas;
};

template <class T, int FLUX, int TP, int TS>
constexpr size_t adj_smem_bytes() {
  constexpr int NH = (TP + 4) * (TS + 4);
  return sizeof(T) * 2 * (SweepLayout<FLUX>::NFF + SweepLayout<FLUX>::NT1) * NH;
}

// Rows of the t1-pass buffer read by the t2 pass for call c = 3 i + r of
// state group s (i the component, r = 0: the value field, which also gives
// the t2-derivative; 1: its t1-derivative; 2: its normal slope) at the t1
// abscissa m1.
template <int NV>
__device__ __forceinline__ int t2_row(int s, int c, int m1) {
  const int k = 5 * s + c / 3, r = c % 3;
  return r == 0 ? 4 * k + m1 : (r == 1 ? 4 * k + 2 + m1 : 4 * NV + 2 * k + m1);
}

// The point-state entries of call c (compile-time) from the tangential
// value v and derivative dv at this thread's t2 abscissa.
template <class T>
__device__ __forceinline__ void t2_assign(PointState<T>& p, int c, T v, T dv, T rh1, T rh2) {
  const int i = c / 3, r = c % 3;
  if (r == 0) {
    p.q[i] = v;
    p.dq[2][i] = dv * rh2;
  } else if (r == 1) {
    p.dq[1][i] = v * rh1;
  } else {
    p.dq[0][i] = v;
  }
}

// Cotangents of the tangential value and derivative of call c (the
// transpose of t2_assign).
template <class T>
__device__ __forceinline__ void t2_cot(const PointState<T>& p, int c, T rh1, T rh2, T& gv, T& gd) {
  const int i = c / 3, r = c % 3;
  gv = r == 0 ? p.q[i] : (r == 1 ? p.dq[1][i] * rh1 : p.dq[0][i]);
  gd = r == 0 ? p.dq[2][i] * rh2 : T(0);
}

template <class T, int MODE, int FLUX, int TP, int TS, int NT>
__global__ void __launch_bounds__(NT) k_sweep_adj(AdjArgs<T> a) {
  constexpr int HP = TP + 4, HS = TS + 4, NH = HP * HS;
  constexpr int NV = SweepLayout<FLUX>::NV;
  constexpr int NFF = SweepLayout<FLUX>::NFF;
  constexpr int NT1 = SweepLayout<FLUX>::NT1;
  constexpr int NS = FLUX == FLUX_FULL ? 3 : 1;
  constexpr int NFACE = TP * TS;
  constexpr int TPF = NT / NFACE;
  static_assert(TPF * NFACE == NT && (TPF == 2 || TPF == 4), "tile must give 2 or 4 threads per face");
  constexpr unsigned kAll = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ff = reinterpret_cast<T*>(smem_raw);  // [NFF][NH] face fields
  T* tb = ff + NFF * NH;                   // [NT1][NH] t1 pass
  T* tbc = tb + NT1 * NH;                  // [NT1][NH] cotangents of the t1 pass
  T* ffc = tbc + NT1 * NH;                 // [NFF][NH] cotangents of the face fields

  const int d = a.d;
  const SweepAxes ax = sweep_axes(d, a.g);
  const int P = ax.P, S = ax.S;
  const bool t1P = ax.t1P;
  const int nP = a.g.n[P], nS = a.g.n[S], nd = a.g.n[d];
  const int p0 = blockIdx.x * TP, s0 = blockIdx.y * TS;
  const int f0 = blockIdx.z * a.chunk;
  const int f1 = min(f0 + a.chunk, nd + 1);
  const int tid = threadIdx.x;
  const T dt = T(a.scal[0]);

  // TPF consecutive threads per face.  Thread tid takes the t2 abscissa
  // m2 = tid & 1 and its neighbour tid ^ 1 (same warp, same face) the other:
  // each tangential reconstruction gives both abscissae, so the pair splits
  // the t2 pass and its transpose between them and swaps halves by shuffles.
  const int face = tid / TPF, sub = tid % TPF;
  const int m2 = sub & 1;
  const int ip = face % TP, is = face / TP;
  const bool f_valid = (p0 + ip < nP) && (s0 + is < nS);
  const int cP = min(p0 + ip, nP - 1), cS = min(s0 + is, nS - 1);
  const int ct1 = t1P ? cP : cS, ct2 = t1P ? cS : cP;
  const T rh1 = T(1) / a.wt1[ct1 + kGhost], rh2 = T(1) / a.wt2[ct2 + kGhost];
  const int at3 = (is + 2) * HP + (ip + 2);
  const int st2 = t1P ? HP : 1;
  const int st1 = t1P ? 1 : HP;
  const int items = t1P ? TP * HS : HP * TS;  // points of the t1 pass

  for (int f = f0; f < f1; ++f) {
    // ---------------- forward: face fields, t1 pass ----------------
    for (int h = tid; h < NH; h += NT) {
      const int hp = h % HP, hs = h / HP;
      const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
      if (Pc <= nP + 1 && Sc <= nS + 1) {
        face_fields_item<T, MODE, FLUX, NH>(a.q, a.g, ax, a.wn, a.gas, f, Pc, Sc, h, ff);
      } else {
#pragma unroll 1
        for (int k = 0; k < NFF; ++k) ff[k * NH + h] = T(0);
      }
#pragma unroll 1
      for (int k = 0; k < NFF; ++k) ffc[k * NH + h] = T(0);
    }
    for (int i = tid; i < NT1 * NH; i += NT) tbc[i] = T(0);
    __syncthreads();
    // One group of five fields per work item (2 NV / 5 groups per point).
    for (int u = tid; u < items * (2 * NV / 5); u += NT) {
      const int it = u % items, grp = u / items;
      const int hp2 = t1P ? 2 + it % TP : it % HP;
      const int hs2 = t1P ? it / TP : 2 + it / HP;
      if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR)
        t1_pass_group_wx2<recon_of<MODE>(), NV, NH>(ff, tb, hs2 * HP + hp2, st1, grp);
      else
        t1_pass_group<T, MODE, NV, NH>(ff, tb, hs2 * HP + hp2, st1, grp);
    }
    __syncthreads();

    // ---------------- R3: flux VJP and transposed t2 pass ----------------
    // Every thread takes part (the pair shuffles); a face outside the grid
    // computes on the tile's padding and adds nothing.
    {
      // Face-flux cotangents from L_c = -(F_{c+1/2} - F_{c-1/2}) / h_c: the face
      // f is the right face of cell f-1 and the left face of cell f.
      T gF[5], gdF[5];
      {
        T cF[5] = {0, 0, 0, 0, 0}, cdF[5] = {0, 0, 0, 0, 0};
        int c[3];
        c[P] = cP;
        c[S] = cS;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int cell = f - 1 + side;
          if (cell < 0 || cell >= nd) continue;
          c[d] = cell;
          const long long ci = ((long long)c[2] * a.g.n[1] + c[1]) * a.g.n[0] + c[0];
          const T sgn = side == 0 ? T(-1) : T(1);
          const T r = sgn / a.wn[cell + kGhost];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            if (a.wL) cF[v] += r * a.wL[v * a.g.N + ci];
            cdF[v] += r * a.wdL[v * a.g.N + ci];
          }
        }
        // Local frame; the face flux is the 1/4-weighted Gauss sum.
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          gF[i] = T(0.25) * cF[ax.gv[i]];
          gdF[i] = T(0.25) * cdF[ax.gv[i]];
        }
      }
#pragma unroll 1
      for (int m1 = sub >> 1; m1 < 2; m1 += TPF / 2) {
        PointState<T> st[NS], ct[NS];
        // Forward t2 pass, one state group per iteration: the 15 calls of a
        // group (5 components x value field, t1-derivative, normal slope) in
        // pairs, the first of each pair on the m2 = 0 thread and the second
        // on its partner; each keeps its own abscissa's result and sends the
        // other's.  The odd last call runs on both.
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
          PointState<T> g0;
          if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR &&
                        FLUX == FLUX_FULL) {
            // FP32 with nonlinear weights, full flux: the thread's calls of
            // pairs j and j + 4 in the halves of one packed evaluation (the
            // smooth-flux tile keeps its two CTAs per SM on the scalar form).
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int a0 = 2 * jj, a1 = 2 * jj + 1;
              const int b0 = 2 * jj + 8, b1 = 2 * jj + 9 < 15 ? 2 * jj + 9 : 2 * jj + 8;
              const T* sa = tb + t2_row<NV>(s, m2 ? a1 : a0, m1) * NH + at3;
              const T* sb = tb + t2_row<NV>(s, m2 ? b1 : b0, m1) * NH + at3;
              float2 f[5], v[2], dv[2];
#pragma unroll
              for (int k = 0; k < 5; ++k) f[k] = make_float2(sa[(k - 2) * st2], sb[(k - 2) * st2]);
              tangential_weno_x2<recon_of<MODE>()>(f[0], f[1], f[2], f[3], f[4], v, dv);
              {
                const T ov = m2 ? v[1].x : v[0].x, od = m2 ? dv[1].x : dv[0].x;
                const T rv = __shfl_xor_sync(kAll, m2 ? v[0].x : v[1].x, 1);
                const T rd = __shfl_xor_sync(kAll, m2 ? dv[0].x : dv[1].x, 1);
                t2_assign(g0, a0, m2 ? rv : ov, m2 ? rd : od, rh1, rh2);
                t2_assign(g0, a1, m2 ? ov : rv, m2 ? od : rd, rh1, rh2);
              }
              {
                const T ov = m2 ? v[1].y : v[0].y, od = m2 ? dv[1].y : dv[0].y;
                const T rv = __shfl_xor_sync(kAll, m2 ? v[0].y : v[1].y, 1);
                const T rd = __shfl_xor_sync(kAll, m2 ? dv[0].y : dv[1].y, 1);
                t2_assign(g0, b0, m2 ? rv : ov, m2 ? rd : od, rh1, rh2);
                if (b1 != b0) t2_assign(g0, b1, m2 ? ov : rv, m2 ? od : rd, rh1, rh2);
              }
            }
          } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c0 = 2 * j, c1 = 2 * j + 1 < 15 ? 2 * j + 1 : 2 * j;
            const T* src = tb + t2_row<NV>(s, m2 ? c1 : c0, m1) * NH + at3;
            T v[2], dv[2];
            tangential<MODE>(src[-2 * st2], src[-st2], src[0], src[st2], src[2 * st2], v, dv);
            const T ov = m2 ? v[1] : v[0], od = m2 ? dv[1] : dv[0];
            const T rv = __shfl_xor_sync(kAll, m2 ? v[0] : v[1], 1);
            const T rd = __shfl_xor_sync(kAll, m2 ? dv[0] : dv[1], 1);
            t2_assign(g0, c0, m2 ? rv : ov, m2 ? rd : od, rh1, rh2);
            if (c1 != c0) t2_assign(g0, c1, m2 ? ov : rv, m2 ? od : rd, rh1, rh2);
          }
          }
          if (s == 0) st[0] = g0;
          else if (NS > 1 && s == 1) st[NS > 1 ? 1 : 0] = g0;
          else if (NS > 2) st[NS > 2 ? 2 : 0] = g0;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            ct[s].q[i] = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) ct[s].dq[c][i] = T(0);
          }
        flux_vjp<T, FLUX>(st, a.gas, dt, a.wL != nullptr, gF, gdF, ct);
        // Transposed t2 pass into the t1-pass cotangents, in the same pairs:
        // the thread that owns a call receives its partner's cotangent of it
        // and transposes the reconstruction for both abscissae at once.
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
          PointState<T> cs = ct[0];
          if (NS > 1 && s == 1) cs = ct[NS > 1 ? 1 : 0];
          if (NS > 2 && s == 2) cs = ct[NS > 2 ? 2 : 0];
          if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR &&
                        FLUX == FLUX_FULL) {
            // The same pairs j and j + 4 as the forward pass, transposed in
            // one packed evaluation.
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int a0 = 2 * jj, a1 = 2 * jj + 1;
              const int b0 = 2 * jj + 8, b1 = 2 * jj + 9 < 15 ? 2 * jj + 9 : 2 * jj + 8;
              T gva[2], gda[2], gvb[2], gdb[2];
              {
                T v0, d0, v1, d1;
                t2_cot(cs, a0, rh1, rh2, v0, d0);
                t2_cot(cs, a1, rh1, rh2, v1, d1);
                const T rv = __shfl_xor_sync(kAll, m2 ? v0 : v1, 1);
                const T rd = __shfl_xor_sync(kAll, m2 ? d0 : d1, 1);
                const T ov = m2 ? v1 : v0, od = m2 ? d1 : d0;
                gva[0] = m2 ? rv : ov;
                gva[1] = m2 ? ov : rv;
                gda[0] = m2 ? rd : od;
                gda[1] = m2 ? od : rd;
              }
              {
                T v0, d0, v1, d1;
                t2_cot(cs, b0, rh1, rh2, v0, d0);
                t2_cot(cs, b1, rh1, rh2, v1, d1);
                const T rv = __shfl_xor_sync(kAll, m2 ? v0 : v1, 1);
                const T rd = __shfl_xor_sync(kAll, m2 ? d0 : d1, 1);
                const T ov = m2 ? v1 : v0, od = m2 ? d1 : d0;
                const bool owner = b1 != b0 || m2 == 0;  // the odd last call: one thread
                gvb[0] = owner ? (m2 ? rv : ov) : T(0);
                gvb[1] = owner ? (m2 ? ov : rv) : T(0);
                gdb[0] = owner ? (m2 ? rd : od) : T(0);
                gdb[1] = owner ? (m2 ? od : rd) : T(0);
              }
              const bool anya = gva[0] != T(0) || gva[1] != T(0) || gda[0] != T(0) || gda[1] != T(0);
              const bool anyb = gvb[0] != T(0) || gvb[1] != T(0) || gdb[0] != T(0) || gdb[1] != T(0);
              if (f_valid && (anya || anyb)) {
                const int rowa = t2_row<NV>(s, m2 ? a1 : a0, m1), rowb = t2_row<NV>(s, m2 ? b1 : b0, m1);
                const T* sa = tb + rowa * NH + at3;
                const T* sb = tb + rowb * NH + at3;
                float2 f[5], cot[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                  f[k] = make_float2(sa[(k - 2) * st2], sb[(k - 2) * st2]);
                  cot[k] = make_float2(0.f, 0.f);
                }
                const float2 gv2[2] = {make_float2(gva[0], gvb[0]), make_float2(gva[1], gvb[1])};
                const float2 gd2[2] = {make_float2(gda[0], gdb[0]), make_float2(gda[1], gdb[1])};
                tangential_vjp_x2<recon_of<MODE>()>(f, gv2, gd2, cot);
                if (anya) {
                  T* dst = tbc + rowa * NH + at3;
#pragma unroll
                  for (int k = 0; k < 5; ++k) atomicAdd(dst + (k - 2) * st2, cot[k].x);
                }
                if (anyb) {
                  T* dst = tbc + rowb * NH + at3;
#pragma unroll
                  for (int k = 0; k < 5; ++k) atomicAdd(dst + (k - 2) * st2, cot[k].y);
                }
              }
            }
          } else
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c0 = 2 * j, c1 = 2 * j + 1 < 15 ? 2 * j + 1 : 2 * j;
            T v0, d0, v1, d1;
            t2_cot(cs, c0, rh1, rh2, v0, d0);
            t2_cot(cs, c1, rh1, rh2, v1, d1);
            const T rv = __shfl_xor_sync(kAll, m2 ? v0 : v1, 1);
            const T rd = __shfl_xor_sync(kAll, m2 ? d0 : d1, 1);
            const T ov = m2 ? v1 : v0, od = m2 ? d1 : d0;
            const T gv[2] = {m2 ? rv : ov, m2 ? ov : rv};
            const T gd[2] = {m2 ? rd : od, m2 ? od : rd};
            const bool owner = c1 != c0 || m2 == 0;
            if (f_valid && owner && (gv[0] != T(0) || gv[1] != T(0) || gd[0] != T(0) || gd[1] != T(0))) {
              const int row = t2_row<NV>(s, m2 ? c1 : c0, m1);
              const T* src = tb + row * NH + at3;
              const T fv[5] = {src[-2 * st2], src[-st2], src[0], src[st2], src[2 * st2]};
              T cot[5] = {0, 0, 0, 0, 0};
              tangential_vjp<MODE>(fv, gv, gd, cot);
              T* dst = tbc + row * NH + at3;
#pragma unroll
              for (int jj = 0; jj < 5; ++jj) atomicAdd(dst + (jj - 2) * st2, cot[jj]);
            }
          }
        }
      }
    }
    __syncthreads();

    // ---------------- R2: transposed t1 pass ----------------
    // One field of one point per work item; FP32 with nonlinear weights: a
    // pair of fields per item, transposed in packed FP32 pairs.
    if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR) {
      for (int u = tid; u < items * NV; u += NT) {
        const int it = u % items, kp = u / items;
        const int hp2 = t1P ? 2 + it % TP : it % HP;
        const int hs2 = t1P ? it / TP : 2 + it / HP;
        const int at = hs2 * HP + hp2;
        float gvs[2][2], gds[2][2];  // [field of the pair][abscissa]
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int k = 2 * kp + e2;
          if (k < NV) {
            gvs[e2][0] = tbc[(4 * k + 0) * NH + at];
            gvs[e2][1] = tbc[(4 * k + 1) * NH + at];
            gds[e2][0] = tbc[(4 * k + 2) * NH + at];
            gds[e2][1] = tbc[(4 * k + 3) * NH + at];
          } else {
            gvs[e2][0] = tbc[(4 * NV + 2 * (k - NV) + 0) * NH + at];
            gvs[e2][1] = tbc[(4 * NV + 2 * (k - NV) + 1) * NH + at];
            gds[e2][0] = gds[e2][1] = 0.f;
          }
        }
        if (gvs[0][0] == 0.f && gvs[0][1] == 0.f && gds[0][0] == 0.f && gds[0][1] == 0.f &&
            gvs[1][0] == 0.f && gvs[1][1] == 0.f && gds[1][0] == 0.f && gds[1][1] == 0.f)
          continue;
        const float2 gv2[2] = {make_float2(gvs[0][0], gvs[1][0]), make_float2(gvs[0][1], gvs[1][1])};
        const float2 gd2[2] = {make_float2(gds[0][0], gds[1][0]), make_float2(gds[0][1], gds[1][1])};
        const T* src0 = ff + (2 * kp) * NH + at;
        const T* src1 = src0 + NH;
        float2 fv[5], cot[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          fv[j] = make_float2(src0[(j - 2) * st1], src1[(j - 2) * st1]);
          cot[j] = make_float2(0.f, 0.f);
        }
        tangential_vjp_x2<recon_of<MODE>()>(fv, gv2, gd2, cot);
        T* dst0 = ffc + (2 * kp) * NH + at;
        T* dst1 = dst0 + NH;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          atomicAdd(dst0 + (j - 2) * st1, cot[j].x);
          atomicAdd(dst1 + (j - 2) * st1, cot[j].y);
        }
      }
    } else
    for (int u = tid; u < items * 2 * NV; u += NT) {
      const int it = u % items, k = u / items;
      const int hp2 = t1P ? 2 + it % TP : it % HP;
      const int hs2 = t1P ? it / TP : 2 + it / HP;
      const int at = hs2 * HP + hp2;
      const bool value_field = k < NV;
      T gv2[2], gd2[2];
      if (value_field) {
        gv2[0] = tbc[(4 * k + 0) * NH + at];
        gv2[1] = tbc[(4 * k + 1) * NH + at];
        gd2[0] = tbc[(4 * k + 2) * NH + at];
        gd2[1] = tbc[(4 * k + 3) * NH + at];
      } else {
        gv2[0] = tbc[(4 * NV + 2 * (k - NV) + 0) * NH + at];
        gv2[1] = tbc[(4 * NV + 2 * (k - NV) + 1) * NH + at];
        gd2[0] = gd2[1] = T(0);
      }
      if (gv2[0] == T(0) && gv2[1] == T(0) && gd2[0] == T(0) && gd2[1] == T(0)) continue;
      const T* src = ff + k * NH + at;
      const T fv[5] = {src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1]};
      T cot[5] = {0, 0, 0, 0, 0};
      tangential_vjp<MODE>(fv, gv2, gd2, cot);
      T* dst = ffc + k * NH + at;
#pragma unroll
      for (int j = 0; j < 5; ++j) atomicAdd(dst + (j - 2) * st1, cot[j]);
    }
    __syncthreads();

    // ---------------- R1: face fields -> cells ----------------
    // R1a, per point: the compatibility state's cotangent onto those of Q_l
    // and Q_r (full flux: added to their face-field cotangents; smooth flux:
    // written to rows 0-9 of the t1 cotangent buffer, free by now).
    T* gql = FLUX == FLUX_FULL ? ffc : tbc;
    for (int h = tid; h < NH; h += NT) {
      const int hp = h % HP, hs = h / HP;
      const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
      if (Pc > nP + 1 || Sc > nS + 1) continue;
      T g0[5], cl[5], cr[5];
      bool any = false;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        g0[i] = ffc[((FLUX == FLUX_FULL ? 10 : 0) + i) * NH + h];
        any = any || g0[i] != T(0);
        cl[i] = FLUX == FLUX_FULL ? ffc[i * NH + h] : T(0);
        cr[i] = FLUX == FLUX_FULL ? ffc[(5 + i) * NH + h] : T(0);
      }
      if (any) {
        T Ql[5], Qr[5];
        if constexpr (FLUX == FLUX_FULL) {
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            Ql[i] = ff[i * NH + h];
            Qr[i] = ff[(5 + i) * NH + h];
          }
        } else {
          int c[3];
          c[d] = f - 3;
          c[P] = Pc;
          c[S] = Sc;
          const long long cb = pad_index(a.g, c[0], c[1], c[2]);
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            const T* qv = a.q + ax.gv[i] * a.g.P + cb;
            T qc[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) qc[k] = qv[k * ax.sd];
            T Li, Ri, Lr, Rr;
            weno5_pair<MODE>(qc[0], qc[1], qc[2], qc[3], qc[4], Li, Ri);
            weno5_pair<MODE>(qc[1], qc[2], qc[3], qc[4], qc[5], Lr, Rr);
            Ql[i] = Ri;
            Qr[i] = Lr;
          }
        }
        compat_vjp(Ql, Qr, g0, a.gas, cl, cr);
      }
      if (any || FLUX != FLUX_FULL) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          gql[i * NH + h] = cl[i];
          gql[(5 + i) * NH + h] = cr[i];
        }
      }
    }
    __syncthreads();
    // R1b, per point and component: the normal slopes and the WENO5 pairs
    // transposed, scattered into the cells f-3 .. f+2.
    {
      const T hl = a.wn[f - 1 + kGhost], hr = a.wn[f + kGhost];
      const T rhl = T(1) / hl, rhr = T(1) / hr, r6 = T(1) / (T(6) * (hl + hr));
      for (int u = tid; u < 5 * NH; u += NT) {
        const int h = u % NH, i = u / NH;
        const int hp = h % HP, hs = h / HP;
        const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
        if (Pc > nP + 1 || Sc > nS + 1) continue;
        const T gQl = gql[i * NH + h], gQr = gql[(5 + i) * NH + h];
        const T gDl = FLUX == FLUX_FULL ? ffc[(15 + i) * NH + h] : T(0);
        const T gDr = FLUX == FLUX_FULL ? ffc[(20 + i) * NH + h] : T(0);
        const T gD0 = ffc[((FLUX == FLUX_FULL ? 25 : 5) + i) * NH + h];
        if (gQl == T(0) && gQr == T(0) && gDl == T(0) && gDr == T(0) && gD0 == T(0)) continue;
        int c[3];
        c[d] = f - 3;
        c[P] = Pc;
        c[S] = Sc;
        const long long cb = pad_index(a.g, c[0], c[1], c[2]);
        const T* qv = a.q + ax.gv[i] * a.g.P + cb;
        T qc[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) qc[k] = qv[k * ax.sd];
        T gq[6] = {0, 0, 0, 0, 0, 0};
        // Slopes: Dl = (4 Ri + 2 Li - 6 q2)/hl, Dr = -(4 Lr + 2 Rr - 6 q3)/hr,
        // D0 = (q1 - 15 q2 + 15 q3 - q4) / (6 (hl + hr)).
        const T gRi = gQl + T(4) * rhl * gDl, gLi = T(2) * rhl * gDl;
        const T gLr = gQr - T(4) * rhr * gDr, gRr = -T(2) * rhr * gDr;
        gq[2] -= T(6) * rhl * gDl;
        gq[3] += T(6) * rhr * gDr;
        gq[1] += r6 * gD0;
        gq[2] -= T(15) * r6 * gD0;
        gq[3] += T(15) * r6 * gD0;
        gq[4] -= r6 * gD0;
        if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR) {
          // both cells' pairs in the halves of packed FP32 pairs
          float2 q2[5], c2[5];
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            q2[j] = make_float2(qc[j], qc[j + 1]);
            c2[j] = make_float2(0.f, 0.f);
          }
          weno5_pair_vjp_x2<recon_of<MODE>()>(q2, make_float2(gLi, gLr), make_float2(gRi, gRr), c2);
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            gq[j] += c2[j].x;
            gq[j + 1] += c2[j].y;
          }
        } else {
          weno5_pair_vjp<MODE>(&qc[0], gLi, gRi, &gq[0]);
          weno5_pair_vjp<MODE>(&qc[1], gLr, gRr, &gq[1]);
        }
        T* accv = a.acc + ax.gv[i] * a.g.P + cb;
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (gq[k] != T(0)) atomicAdd(accv + k * ax.sd, gq[k]);
      }
    }
    __syncthreads();
  }
}

// Returns the cotangents collected on ghost cells to their periodic images,
// in the reverse order of the ghost fill (z, then y, then x).  Wall
// boundaries are not handled (the adjoint rejects them).
template <class T>
__global__ void k_fold_ghosts_z(T* __restrict__ acc, GridDev g) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long plane = (long long)g.p[0] * g.p[1];
  if (tid >= 6 * plane) return;
  const long long xy = tid % plane;
  const int m = int(tid / plane);
  const int z = m < 3 ? -1 - m : g.n[2] + (m - 3);
  const int src = m < 3 ? g.n[2] - 1 - m : m - 3;
  const long long gi = (long long)(z + kGhost) * plane + xy;
  const long long si = (long long)(src + kGhost) * plane + xy;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    acc[v * g.P + si] += acc[v * g.P + gi];
    acc[v * g.P + gi] = T(0);
  }
}
template <class T>
__global__ void k_fold_ghosts_y(T* __restrict__ acc, GridDev g) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= 6LL * g.p[0] * g.n[2]) return;
  const int x = int(tid % g.p[0]) - kGhost;
  const long long r = tid / g.p[0];
  const int m = int(r % 6), z = int(r / 6);
  const int y = m < 3 ? -1 - m : g.n[1] + (m - 3);
  const int src = m < 3 ? g.n[1] - 1 - m : m - 3;
  const long long gi = pad_index(g, x, y, z), si = pad_index(g, x, src, z);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    acc[v * g.P + si] += acc[v * g.P + gi];
    acc[v * g.P + gi] = T(0);
  }
}
template <class T>
__global__ void k_fold_ghosts_x(T* __restrict__ acc, GridDev g) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= 6LL * g.n[1] * g.n[2]) return;
  const int m = int(tid % 6);
  const long long r = tid / 6;
  const int y = int(r % g.n[1]), z = int(r / g.n[1]);
  const int x = m < 3 ? -1 - m : g.n[0] + (m - 3);
  const int src = m < 3 ? g.n[0] - 1 - m : m - 3;
  const long long gi = pad_index(g, x, y, z), si = pad_index(g, src, y, z);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    acc[v * g.P + si] += acc[v * g.P + gi];
    acc[v * g.P + gi] = T(0);
  }
}

// Elementwise pieces of the step's adjoint (interior cells, [5][N]):
// mode 0: wdL = c1 * lam                      (the Q* evaluation; wL = 0)
// mode 1: wL = dt lam + dt/2 mu, wdL = dt^2/6 lam + dt^2/8 mu, mu = acc
// mode 2: out = lam + mu_star + acc           (FP64 result)
template <class T>
__global__ void k_adj_combine(int mode, const double* __restrict__ lam, const T* __restrict__ acc,
                              T* __restrict__ mu_star, T* __restrict__ wL, T* __restrict__ wdL,
                              double* __restrict__ out, const double* __restrict__ scal, GridDev g) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const double dt = scal[0];
  const int nx = g.n[0], ny = g.n[1];
  const int x = int(c % nx);
  const long long r = c / nx;
  const int y = int(r % ny), z = int(r / ny);
  const long long pi = pad_index(g, x, y, z);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double l = lam[v * g.N + c];
    if (mode == 0) {
      wdL[v * g.N + c] = T(dt * dt / 3.0 * l);
    } else if (mode == 1) {
      const double m = double(acc[v * g.P + pi]);
      mu_star[v * g.N + c] = T(m);
      wL[v * g.N + c] = T(dt * l + 0.5 * dt * m);
      wdL[v * g.N + c] = T(dt * dt / 6.0 * l + dt * dt / 8.0 * m);
    } else {
      out[v * g.N + c] = l + double(mu_star[v * g.N + c]) + double(acc[v * g.P + pi]);
    }
  }
}

}  // namespace hgks

// Reverse-mode derivatives (vector-Jacobian products) of the fluxes at one
// Gauss point with respect to their input states, values q and slopes dq
// together, in one backward pass per part: the half-space parts of the full
// flux (flux_full_side), its equilibrium part (flux_full_eq), the full flux
// assembled from them with the collision time and the fit of Eq. (7)
// (flux_full_vjp), the smooth flux (flux_smooth_rev) and the sign moments of
// the compatibility state.  Every function is the transpose of the forward
// function it names, with the forward intermediates recomputed; the
// slopes enter each part linearly, through the same intermediates as the
// values, so their cotangents come out of the same pass.  No counterpart in
// the paper.
#pragma once

#include "dual.cuh"
#include "physics.cuh"

namespace hgks {

// Cotangents of the fields of Prim.
template <class T>
struct PrimBar {
  T rho, inv, U, V, W, dp, p, lam, theta;
};

template <class T>
HGKS_HD void prim_bar_zero(PrimBar<T>& b) {
  b.rho = b.inv = b.U = b.V = b.W = b.dp = b.p = b.lam = b.theta = T(0);
}

// prim_of transposed: b holds the cotangents of the fields of s = prim_of(q);
// adds the cotangent of q to qb.
template <class T>
HGKS_HD void prim_of_rev(const T q[5], const Prim<T>& s, const Gas<T>& g, PrimBar<T> b, T qb[5]) {
  // lam = 1/(2 theta)
  b.theta += b.lam * (-T(0.5) / (s.theta * s.theta));
  // theta = p inv
  b.p += b.theta * s.inv_rho;
  b.inv += b.theta * s.p;
  // p = p_r + dp
  b.dp += b.p;
  // dp = gm1 (q4 - (q1 U + q2 V + q3 W)/2)
  const T h = g.gm1 * b.dp;
  qb[4] += h;
  qb[1] += -T(0.5) * h * s.U;
  qb[2] += -T(0.5) * h * s.V;
  qb[3] += -T(0.5) * h * s.W;
  b.U += -T(0.5) * h * q[1];
  b.V += -T(0.5) * h * q[2];
  b.W += -T(0.5) * h * q[3];
  // U = q1 inv, V = q2 inv, W = q3 inv
  qb[1] += b.U * s.inv_rho;
  qb[2] += b.V * s.inv_rho;
  qb[3] += b.W * s.inv_rho;
  b.inv += b.U * q[1] + b.V * q[2] + b.W * q[3];
  // inv = 1/rho, rho = rho_r + q0
  b.rho += -b.inv * s.inv_rho * s.inv_rho;
  qb[0] += b.rho;
}

// slope_solve transposed: a = slope_solve(s, b); given ab (cotangent of a)
// adds to sb (the state's fields) and bb (cotangent of b).
template <class T>
HGKS_HD void slope_solve_rev(const Prim<T>& s, const Gas<T>& g, const T b[5], const T ab[5],
                             PrimBar<T>& sb, T bb[5]) {
  const T U = s.U, V = s.V, W = s.W;
  const T q2 = U * U + V * V + W * W;
  const T k3t = (g.K + T(3)) * s.theta;
  const T l2 = T(2) * s.lam;
  const T c4 = l2 * l2 / (g.K + T(3));
  const T t = T(2) * (b[4] - U * b[1] - V * b[2] - W * b[3]) + (q2 - k3t) * b[0];
  const T a4 = c4 * t;
  const T a3 = l2 * (b[3] - W * b[0]) - W * a4;
  const T a2 = l2 * (b[2] - V * b[0]) - V * a4;
  const T a1 = l2 * (b[1] - U * b[0]) - U * a4;
  // a0 = b0 - U a1 - V a2 - W a3 - a4 (q2 + k3t)/2
  T a1b = ab[1] - ab[0] * U, a2b = ab[2] - ab[0] * V, a3b = ab[3] - ab[0] * W;
  T a4b = ab[4] - T(0.5) * ab[0] * (q2 + k3t);
  T Ub = -ab[0] * a1, Vb = -ab[0] * a2, Wb = -ab[0] * a3;
  T q2b = -T(0.5) * ab[0] * a4, k3tb = -T(0.5) * ab[0] * a4;
  bb[0] += ab[0];
  // a_i = l2 (b_i - U_i b0) - U_i a4, i = 1, 2, 3
  T l2b = a1b * (b[1] - U * b[0]) + a2b * (b[2] - V * b[0]) + a3b * (b[3] - W * b[0]);
  bb[1] += a1b * l2;
  bb[2] += a2b * l2;
  bb[3] += a3b * l2;
  bb[0] += -l2 * (a1b * U + a2b * V + a3b * W);
  Ub += -a1b * (l2 * b[0] + a4);
  Vb += -a2b * (l2 * b[0] + a4);
  Wb += -a3b * (l2 * b[0] + a4);
  a4b += -(a1b * U + a2b * V + a3b * W);
  // a4 = c4 t
  const T c4b = a4b * t, tb = a4b * c4;
  // t = 2 (b4 - U b1 - V b2 - W b3) + (q2 - k3t) b0
  bb[4] += T(2) * tb;
  bb[1] += -T(2) * tb * U;
  bb[2] += -T(2) * tb * V;
  bb[3] += -T(2) * tb * W;
  bb[0] += tb * (q2 - k3t);
  Ub += -T(2) * tb * b[1];
  Vb += -T(2) * tb * b[2];
  Wb += -T(2) * tb * b[3];
  q2b += tb * b[0];
  k3tb += -tb * b[0];
  // c4 = l2^2/(K+3), l2 = 2 lam, k3t = (K+3) theta, q2 = |U|^2
  l2b += c4b * T(2) * l2 / (g.K + T(3));
  sb.lam += T(2) * l2b;
  sb.theta += (g.K + T(3)) * k3tb;
  sb.U += Ub + T(2) * U * q2b;
  sb.V += Vb + T(2) * V * q2b;
  sb.W += Wb + T(2) * W * q2b;
}

// euler_jvp<J> transposed in the state (dQ held fixed): out = J_J(Q) dQ;
// given ob adds to sb and Hb.
template <int J, class T>
HGKS_HD void euler_jvp_rev_state(const Prim<T>& s, T H, const T dQ[5], const Gas<T>& g,
                                 const T ob[5], PrimBar<T>& sb, T& Hb) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
  T du[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) du[i] = (dQ[1 + i] - U[i] * dQ[0]) * inv;
  const T dp = g.gm1 * (dQ[4] - U[0] * dQ[1] - U[1] * dQ[2] - U[2] * dQ[3] +
                        T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) * dQ[0]);
  const T mJ = s.rho * U[J];
  T Ub[3] = {T(0), T(0), T(0)}, dub[3] = {T(0), T(0), T(0)};
  T mJb = T(0), dpb = T(0);
  // out[1+i] = dQ[1+J] U_i + mJ du_i (+ dp for i = J)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[i] += ob[1 + i] * dQ[1 + J];
    mJb += ob[1 + i] * du[i];
    dub[i] += ob[1 + i] * mJ;
  }
  dpb += ob[1 + J];
  // out4 = du_J H + U_J (dQ4 + dp)
  dub[J] += ob[4] * H;
  Hb += ob[4] * du[J];
  Ub[J] += ob[4] * (dQ[4] + dp);
  dpb += ob[4] * U[J];
  // mJ = rho U_J
  sb.rho += mJb * U[J];
  Ub[J] += mJb * s.rho;
  // dp = gm1 (dQ4 - U.dQm + |U|^2/2 dQ0)
#pragma unroll
  for (int i = 0; i < 3; ++i) Ub[i] += dpb * g.gm1 * (U[i] * dQ[0] - dQ[1 + i]);
  // du_i = (dQ[1+i] - U_i dQ0) inv
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[i] += -dub[i] * dQ[0] * inv;
    sb.inv += dub[i] * (dQ[1 + i] - U[i] * dQ[0]);
  }
  sb.U += Ub[0];
  sb.V += Ub[1];
  sb.W += Ub[2];
}

// Cotangents of the normalised moments of Mom.
template <class T>
struct MomBar {
  T u[7], v[7], w[7];
  T xi1, xi2;
};

template <int A, int B, int C, class T>
HGKS_HD void mm_rev(const Mom<T>& m, T bar, MomBar<T>& mb) {
  mb.u[A] += bar * m.v[B] * m.w[C];
  mb.v[B] += bar * m.u[A] * m.w[C];
  mb.w[C] += bar * m.u[A] * m.v[B];
}

// mom_psipsi<A,B,C> transposed: Mb (cotangents of the 15 entries) into mb.
template <int A, int B, int C, class T>
HGKS_HD void mom_psipsi_rev(const Mom<T>& m, const T Mb[15], MomBar<T>& mb) {
  const T x1 = m.xi1, x2 = m.xi2;
  const T m0 = mm<A, B, C>(m);
  const T mu1 = mm<A + 1, B, C>(m), mv1 = mm<A, B + 1, C>(m), mw1 = mm<A, B, C + 1>(m);
  const T mu2 = mm<A + 2, B, C>(m), mv2 = mm<A, B + 2, C>(m), mw2 = mm<A, B, C + 2>(m);
  T m0b = Mb[0], mu1b = Mb[1], mv1b = Mb[2], mw1b = Mb[3];
  T mu2b = Mb[5], mv2b = Mb[9], mw2b = Mb[12];
  T x1b = T(0), x2b = T(0);
  // M[4] = (mu2 + mv2 + mw2 + m0 x1)/2
  {
    const T h = T(0.5) * Mb[4];
    mu2b += h;
    mv2b += h;
    mw2b += h;
    m0b += h * x1;
    x1b += h * m0;
  }
  mm_rev<A + 1, B + 1, C>(m, Mb[6], mb);
  mm_rev<A + 1, B, C + 1>(m, Mb[7], mb);
  // M[8] = (u^3 + u v^2 + u w^2 + mu1 x1)/2
  {
    const T h = T(0.5) * Mb[8];
    mm_rev<A + 3, B, C>(m, h, mb);
    mm_rev<A + 1, B + 2, C>(m, h, mb);
    mm_rev<A + 1, B, C + 2>(m, h, mb);
    mu1b += h * x1;
    x1b += h * mu1;
  }
  mm_rev<A, B + 1, C + 1>(m, Mb[10], mb);
  {
    const T h = T(0.5) * Mb[11];
    mm_rev<A + 2, B + 1, C>(m, h, mb);
    mm_rev<A, B + 3, C>(m, h, mb);
    mm_rev<A, B + 1, C + 2>(m, h, mb);
    mv1b += h * x1;
    x1b += h * mv1;
  }
  {
    const T h = T(0.5) * Mb[13];
    mm_rev<A + 2, B, C + 1>(m, h, mb);
    mm_rev<A, B + 2, C + 1>(m, h, mb);
    mm_rev<A, B, C + 3>(m, h, mb);
    mw1b += h * x1;
    x1b += h * mw1;
  }
  // M[14] = (u4 + v4 + w4 + 2(u2v2 + u2w2 + v2w2) + 2 x1 (mu2 + mv2 + mw2) + x2 m0)/4
  {
    const T h = T(0.25) * Mb[14];
    mm_rev<A + 4, B, C>(m, h, mb);
    mm_rev<A, B + 4, C>(m, h, mb);
    mm_rev<A, B, C + 4>(m, h, mb);
    mm_rev<A + 2, B + 2, C>(m, T(2) * h, mb);
    mm_rev<A + 2, B, C + 2>(m, T(2) * h, mb);
    mm_rev<A, B + 2, C + 2>(m, T(2) * h, mb);
    x1b += T(2) * h * (mu2 + mv2 + mw2);
    mu2b += T(2) * h * x1;
    mv2b += T(2) * h * x1;
    mw2b += T(2) * h * x1;
    x2b += h * m0;
    m0b += h * x2;
  }
  mm_rev<A, B, C>(m, m0b, mb);
  mm_rev<A + 1, B, C>(m, mu1b, mb);
  mm_rev<A, B + 1, C>(m, mv1b, mb);
  mm_rev<A, B, C + 1>(m, mw1b, mb);
  mm_rev<A + 2, B, C>(m, mu2b, mb);
  mm_rev<A, B + 2, C>(m, mv2b, mb);
  mm_rev<A, B, C + 2>(m, mw2b, mb);
  mb.xi1 += x1b;
  mb.xi2 += x2b;
}

// out = M a (sym5_matvec_add) transposed: adds the cotangents of the 15
// stored entries of the symmetric M and of a, given ob.
template <class T>
HGKS_HD void sym5_matvec_rev(const T M[15], const T a[5], const T ob[5], T Mb[15], T ab[5]) {
  // index of the stored entry (i <= j)
  constexpr int idx[5][5] = {{0, 1, 2, 3, 4}, {1, 5, 6, 7, 8}, {2, 6, 9, 10, 11}, {3, 7, 10, 12, 13},
                             {4, 8, 11, 13, 14}};
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      Mb[idx[i][j]] += ob[i] * a[j];
      ab[j] += ob[i] * M[idx[i][j]];
    }
}

// gauss_recursion transposed (m[n+2] = U m[n+1] + (n+1) theta m[n]).
template <class T>
HGKS_HD void gauss_recursion_rev(const T* m, T U, T theta, T* mb, T& Ub, T& thb) {
#pragma unroll
  for (int n = 4; n >= 0; --n) {
    const T b = mb[n + 2];
    Ub += b * m[n + 1];
    mb[n + 1] += b * U;
    thb += b * T(n + 1) * m[n];
    mb[n] += b * T(n + 1) * theta;
  }
}

// moments(s, half = +-1) transposed into sb.
template <class T>
HGKS_HD void moments_rev(const Prim<T>& s, const Gas<T>& g, int half, const Mom<T>& m, MomBar<T> mb,
                         PrimBar<T>& sb) {
  sb.theta += mb.xi1 * g.K + mb.xi2 * g.K * (g.K + T(2)) * T(2) * s.theta;
  T Ub = T(0), Vb = T(0), Wb = T(0), thb = T(0);
  gauss_recursion_rev(m.w, s.W, s.theta, mb.w, Wb, thb);
  Wb += mb.w[1];
  gauss_recursion_rev(m.v, s.V, s.theta, mb.v, Vb, thb);
  Vb += mb.v[1];
  gauss_recursion_rev(m.u, s.U, s.theta, mb.u, Ub, thb);
  // half line: u0 = (1 + sg erf(x))/2, u1 = U u0 + sg e,
  // x = sqrt(lam) U, e = exp(-x^2) / (2 sqrt(pi) sqrt(lam))
  const T sl = tsqrt(s.lam);
  const T x = sl * s.U;
  const T ex = texp(-x * x);
  const T e = ex * T(0.28209479177387814) / sl;
  const T sg = T(half);
  Ub += mb.u[1] * m.u[0];
  T u0b = mb.u[0] + mb.u[1] * s.U;
  const T eb = mb.u[1] * sg;
  T xb = eb * e * (-T(2) * x) + u0b * T(0.5) * sg * T(1.1283791670955126) * ex;
  T slb = -eb * e / sl + xb * s.U;
  Ub += xb * sl;
  sb.lam += slb * T(0.5) / sl;
  sb.U += Ub;
  sb.V += Vb;
  sb.W += Wb;
  sb.theta += thb;
}

// euler_jvp<J> transposed in dQ (the state held fixed): adds J_J(Q)^T ob to dQb.
template <int J, class T>
HGKS_HD void euler_jvp_rev_dq(const Prim<T>& s, T H, const Gas<T>& g, const T ob[5], T dQb[5]) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
  const T mJ = s.rho * U[J];
  T dub[3] = {T(0), T(0), T(0)};
  T dpb = T(0);
  dQb[1 + J] += ob[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dQb[1 + J] += ob[1 + i] * U[i];
    dub[i] += ob[1 + i] * mJ;
  }
  dpb += ob[1 + J];
  dub[J] += ob[4] * H;
  dQb[4] += ob[4] * U[J];
  dpb += ob[4] * U[J];
  // dp = gm1 (dQ4 - U.dQm + |U|^2/2 dQ0)
  const T h = g.gm1 * dpb;
  dQb[4] += h;
#pragma unroll
  for (int k = 0; k < 3; ++k) dQb[1 + k] += -h * U[k];
  dQb[0] += h * T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
  // du_i = (dQ[1+i] - U_i dQ0) inv
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dQb[1 + i] += dub[i] * inv;
    dQb[0] += -dub[i] * U[i] * inv;
  }
}

// Cotangents of the values q and slopes dq of the state of flux_full_side
// (side 0: u > 0, side 1: u < 0) as it enters the full flux through the
// fit weights w_k = Fq[k] (F) and dFq[k] (dF) of its three moment vectors V_k
// (flux_full_combine), given the flux cotangents gF, gdF; added to cot.  The
// weights are dual numbers carrying d/dtau; returns the part's share of
// gF . dF/dtau + gdF . d(dF)/dtau.  The cotangent of its pressure (through
// tau) is applied by pressure_viscosity_rev.  The four moment matrices are
// formed one at a time, forward and again backward, to keep few values live.
template <class T>
HGKS_HD T flux_full_side_rev(const PointState<T>& st, const Gas<T>& g, int side, const T gF[5],
                             const T gdF[5], const Dual<T> Fq[3], const Dual<T> dFq[3], PointState<T>& cot) {
  const Prim<T> s = prim_of(st.q, g);
  const T inv = s.inv_rho;
  // forward: slopes a_d = slope_solve(s, dq_d inv), Q_t, A = slope_solve(s, Q_t inv)
  T a[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T bd[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) bd[i] = st.dq[d][i] * inv;
    slope_solve(s, g, bd, a[d]);
  }
  const T H = g.h_r + st.q[4] + s.dp;
  T Qt[5];
  state_time_derivative(s, H, st.dq, g, Qt);
  T bA[5], A[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) bA[i] = Qt[i] * inv;
  slope_solve(s, g, bA, A);
  const int half = side == 0 ? +1 : -1;
  Mom<T> mh;
  moments(s, g, half, mh);
  // V0 = rho <u psi> (the first column of M1), V1 = rho ua, V2 = rho uA with
  // M1 = <u psi psi^T>, uA = M1 A, ua = sum_d <u u_d psi psi^T> a_d.
  T m1[5], ua[5] = {0, 0, 0, 0, 0}, uA[5] = {0, 0, 0, 0, 0};
  {
    T M[15];
    mom_psipsi<1, 0, 0>(mh, M);
#pragma unroll
    for (int i = 0; i < 5; ++i) m1[i] = M[i];
    sym5_matvec_add(M, A, uA);
  }
  {
    T M[15];
    mom_psipsi<2, 0, 0>(mh, M);
    sym5_matvec_add(M, a[0], ua);
  }
  {
    T M[15];
    mom_psipsi<1, 1, 0>(mh, M);
    sym5_matvec_add(M, a[1], ua);
  }
  {
    T M[15];
    mom_psipsi<1, 0, 1>(mh, M);
    sym5_matvec_add(M, a[2], ua);
  }
  // backward: the cotangents of V_k are gV_k = gF w_k + gdF dw_k
  PrimBar<T> sb;
  prim_bar_zero(sb);
  T phi = T(0), uab[5], uAb[5], m1b[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const T gv0 = gF[i] * Fq[0].v + gdF[i] * dFq[0].v, gt0 = gF[i] * Fq[0].d + gdF[i] * dFq[0].d;
    const T gv1 = gF[i] * Fq[1].v + gdF[i] * dFq[1].v, gt1 = gF[i] * Fq[1].d + gdF[i] * dFq[1].d;
    const T gv2 = gF[i] * Fq[2].v + gdF[i] * dFq[2].v, gt2 = gF[i] * Fq[2].d + gdF[i] * dFq[2].d;
    phi += s.rho * (gt0 * m1[i] + gt1 * ua[i] + gt2 * uA[i]);
    sb.rho += gv0 * m1[i] + gv1 * ua[i] + gv2 * uA[i];
    m1b[i] = s.rho * gv0;
    uab[i] = s.rho * gv1;
    uAb[i] = s.rho * gv2;
  }
  MomBar<T> mb;
#pragma unroll
  for (int n = 0; n < 7; ++n) mb.u[n] = mb.v[n] = mb.w[n] = T(0);
  mb.xi1 = mb.xi2 = T(0);
  T Ab[5] = {0, 0, 0, 0, 0}, ab[3][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
  {
    T M[15], Mb[15];
    mom_psipsi<1, 0, 0>(mh, M);
#pragma unroll
    for (int k = 0; k < 15; ++k) Mb[k] = k < 5 ? m1b[k] : T(0);
    sym5_matvec_rev(M, A, uAb, Mb, Ab);
    mom_psipsi_rev<1, 0, 0>(mh, Mb, mb);
  }
  {
    T M[15], Mb[15];
    mom_psipsi<2, 0, 0>(mh, M);
#pragma unroll
    for (int k = 0; k < 15; ++k) Mb[k] = T(0);
    sym5_matvec_rev(M, a[0], uab, Mb, ab[0]);
    mom_psipsi_rev<2, 0, 0>(mh, Mb, mb);
  }
  {
    T M[15], Mb[15];
    mom_psipsi<1, 1, 0>(mh, M);
#pragma unroll
    for (int k = 0; k < 15; ++k) Mb[k] = T(0);
    sym5_matvec_rev(M, a[1], uab, Mb, ab[1]);
    mom_psipsi_rev<1, 1, 0>(mh, Mb, mb);
  }
  {
    T M[15], Mb[15];
    mom_psipsi<1, 0, 1>(mh, M);
#pragma unroll
    for (int k = 0; k < 15; ++k) Mb[k] = T(0);
    sym5_matvec_rev(M, a[2], uab, Mb, ab[2]);
    mom_psipsi_rev<1, 0, 1>(mh, Mb, mb);
  }
  moments_rev(s, g, half, mh, mb, sb);
  // A = slope_solve(s, Q_t inv), Q_t = -sum_d J_d(Q) dq_d
  T bAb[5] = {0, 0, 0, 0, 0};
  slope_solve_rev(s, g, bA, Ab, sb, bAb);
  T nQtb[5], Hb = T(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    nQtb[i] = -bAb[i] * inv;
    sb.inv += bAb[i] * Qt[i];
  }
  // Q_t = -(J_0 dq_0 + J_1 dq_1 + J_2 dq_2): both the state and the slopes
  euler_jvp_rev_state<0>(s, H, st.dq[0], g, nQtb, sb, Hb);
  euler_jvp_rev_state<1>(s, H, st.dq[1], g, nQtb, sb, Hb);
  euler_jvp_rev_state<2>(s, H, st.dq[2], g, nQtb, sb, Hb);
  euler_jvp_rev_dq<0>(s, H, g, nQtb, cot.dq[0]);
  euler_jvp_rev_dq<1>(s, H, g, nQtb, cot.dq[1]);
  euler_jvp_rev_dq<2>(s, H, g, nQtb, cot.dq[2]);
  // H = h_r + q4 + dp
  cot.q[4] += Hb;
  sb.dp += Hb;
  // a_d = slope_solve(s, dq_d inv)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T bd[5], bdb[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 5; ++i) bd[i] = st.dq[d][i] * inv;
    slope_solve_rev(s, g, bd, ab[d], sb, bdb);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      sb.inv += bdb[i] * st.dq[d][i];
      cot.dq[d][i] += bdb[i] * inv;
    }
  }
  prim_of_rev(st.q, s, g, sb, cot.q);
  return phi;
}

// ns_viscous_flux transposed in the state and the viscosity (dq held fixed):
// given Fvb adds to sb and mub.
template <class T>
HGKS_HD void ns_viscous_flux_rev(const Prim<T>& s, const T dq[3][5], const Gas<T>& g, T mu, T heat_scale,
                                 const T Fvb[5], PrimBar<T>& sb, T& mub) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
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
  const T c2 = T(2) / (g.K + T(3));
  const T s00 = mu * (T(2) * du0[0] - c2 * divU);
  const T s01 = mu * (du0[1] + du10);
  const T s02 = mu * (du0[2] + du20);
  const T ch = heat_scale * T(0.5) * (g.K + T(5));
  T Ub[3] = {T(0), T(0), T(0)};
  // Fv = (0, -s00, -s01, -s02, -(s00 U0 + s01 U1 + s02 U2) - ch mu dT0)
  const T s00b = -Fvb[1] - Fvb[4] * U[0];
  const T s01b = -Fvb[2] - Fvb[4] * U[1];
  const T s02b = -Fvb[3] - Fvb[4] * U[2];
  Ub[0] += -Fvb[4] * s00;
  Ub[1] += -Fvb[4] * s01;
  Ub[2] += -Fvb[4] * s02;
  mub += -Fvb[4] * ch * dT0;
  const T dT0b = -Fvb[4] * ch * mu;
  mub += s00b * (T(2) * du0[0] - c2 * divU) + s01b * (du0[1] + du10) + s02b * (du0[2] + du20);
  T du0b[3] = {s00b * mu * T(2), s01b * mu, s02b * mu};
  const T du10b = s01b * mu, du20b = s02b * mu;
  const T divUb = -s00b * mu * c2;
  du0b[0] += divUb;
  const T du11b = divUb, du22b = divUb;
  // dT0 = (dp0 - theta dq00) inv
  const T dp0b = dT0b * inv;
  sb.theta += -dT0b * dq[0][0] * inv;
  sb.inv += dT0b * (dp0 - s.theta * dq[0][0]);
#pragma unroll
  for (int i = 0; i < 3; ++i) Ub[i] += dp0b * g.gm1 * (U[i] * dq[0][0] - dq[0][1 + i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[i] += -du0b[i] * dq[0][0] * inv;
    sb.inv += du0b[i] * (dq[0][1 + i] - U[i] * dq[0][0]);
  }
  Ub[0] += -du10b * dq[1][0] * inv;
  sb.inv += du10b * (dq[1][1] - U[0] * dq[1][0]);
  Ub[1] += -du11b * dq[1][0] * inv;
  sb.inv += du11b * (dq[1][2] - U[1] * dq[1][0]);
  Ub[0] += -du20b * dq[2][0] * inv;
  sb.inv += du20b * (dq[2][1] - U[0] * dq[2][0]);
  Ub[2] += -du22b * dq[2][0] * inv;
  sb.inv += du22b * (dq[2][3] - U[2] * dq[2][0]);
  sb.U += Ub[0];
  sb.V += Ub[1];
  sb.W += Ub[2];
}

// euler_flux_dev transposed: E = (m, m U + dp, m V, m W, U (h_r + q4 + dp)),
// m = rho U; given gE adds to sb and qb.
template <class T>
HGKS_HD void euler_flux_dev_rev(const Prim<T>& s, const T q[5], const Gas<T>& g, const T gE[5],
                                PrimBar<T>& sb, T qb[5]) {
  const T m = s.rho * s.U;
  const T mb = gE[0] + gE[1] * s.U + gE[2] * s.V + gE[3] * s.W;
  sb.U += gE[1] * m + gE[4] * (g.h_r + q[4] + s.dp);
  sb.V += gE[2] * m;
  sb.W += gE[3] * m;
  sb.dp += gE[1] + gE[4] * s.U;
  qb[4] += gE[4] * s.U;
  sb.rho += mb * s.U;
  sb.U += mb * s.rho;
}

// sign_moments transposed (the half-space sign moments S of the
// compatibility state): given gS adds the cotangent of dq to qb.
template <class T>
HGKS_HD void sign_moments_rev(const T dq[5], const Gas<T>& g, const T gS[5], T qb[5]) {
  const Prim<T> s = prim_of(dq, g);
  const T sl = tsqrt(s.lam);
  const T x = sl * s.U;
  const T D0 = terf(x);
  const T ex = texp(-x * x);
  const T R = tsqrt(s.theta + s.theta);
  const T c = T(0.5641895835477563);  // 1/sqrt(pi)
  const T D1 = s.U * D0 + ex * c * R;
  const T D2 = s.U * D1 + s.theta * D0;
  const T G = s.V * s.V + s.W * s.W + (g.K + T(2)) * s.theta;
  PrimBar<T> sb;
  prim_bar_zero(sb);
  const T h = T(0.5) * gS[4];
  sb.rho += gS[0] * D0 + gS[1] * D1 + gS[2] * s.V * D0 + gS[3] * s.W * D0 + h * (D2 + D0 * G);
  T D0b = gS[0] * s.rho + gS[2] * s.rho * s.V + gS[3] * s.rho * s.W + h * s.rho * G;
  T D1b = gS[1] * s.rho;
  const T D2b = h * s.rho;
  sb.V += gS[2] * s.rho * D0 + h * s.rho * D0 * T(2) * s.V;
  sb.W += gS[3] * s.rho * D0 + h * s.rho * D0 * T(2) * s.W;
  sb.theta += h * s.rho * D0 * (g.K + T(2));
  // D2 = U D1 + theta D0
  sb.U += D2b * D1;
  D1b += D2b * s.U;
  sb.theta += D2b * D0;
  D0b += D2b * s.theta;
  // D1 = U D0 + exp(-x^2) R / sqrt(pi), R = sqrt(2 theta)
  sb.U += D1b * D0;
  D0b += D1b * s.U;
  const T exb = D1b * c * R;
  sb.theta += D1b * ex * c / R;
  // ex = exp(-x^2), D0 = erf(x), x = sqrt(lam) U
  const T xb = exb * ex * (-T(2) * x) + D0b * T(2) * c * ex;
  sb.U += xb * sl;
  sb.lam += xb * s.U * T(0.5) / sl;
  prim_of_rev(dq, s, g, sb, qb);
}

// c0 += cotangent of dq along n from tb, the cotangent of the temperature
// slope dT0 = (dp0 - theta dq[0])/rho, dp0 = (gamma-1)(dq[4] - U.dm + |U|^2/2 dq[0]).
template <class T>
HGKS_HD void temperature_slope_vjp(const Prim<T>& s, const Gas<T>& g, T tb, T c0[5]) {
  const T inv = s.inv_rho;
  const T dpb = tb * inv * g.gm1;
  const T q2 = s.U * s.U + s.V * s.V + s.W * s.W;
  c0[0] += -s.theta * tb * inv + T(0.5) * q2 * dpb;
  c0[1] -= s.U * dpb;
  c0[2] -= s.V * dpb;
  c0[3] -= s.W * dpb;
  c0[4] += dpb;
}

// cd += (d Fv / d dq)^T w for ns_viscous_flux (linear in dq).
template <class T>
HGKS_HD void ns_viscous_vjp(const Prim<T>& s, const Gas<T>& g, T mu, T heat_scale, const T w[5],
                           T cd[3][5]) {
  const T inv = s.inv_rho;
  const T U[3] = {s.U, s.V, s.W};
  const T s00 = -w[1] - w[4] * U[0], s01 = -w[2] - w[4] * U[1], s02 = -w[3] - w[4] * U[2];
  const T divb = -mu * T(2) / (g.K + T(3)) * s00;
  const T du0b[3] = {T(2) * mu * s00 + divb, mu * s01, mu * s02};
  const T du10 = mu * s01, du20 = mu * s02, du11 = divb, du22 = divb;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cd[0][1 + i] += du0b[i] * inv;
    cd[0][0] -= U[i] * du0b[i] * inv;
  }
  cd[1][1] += du10 * inv;
  cd[1][2] += du11 * inv;
  cd[1][0] -= (U[0] * du10 + U[1] * du11) * inv;
  cd[2][1] += du20 * inv;
  cd[2][3] += du22 * inv;
  cd[2][0] -= (U[0] * du20 + U[2] * du22) * inv;
  temperature_slope_vjp(s, g, -w[4] * heat_scale * mu * T(0.5) * (g.K + T(5)), cd[0]);
}

// Cotangents of the values q and slopes dq of the state of the smooth flux
// (flux_smooth) given the cotangents gF of F (if want_F) and gdF of dF;
// added to cot.
template <class T>
HGKS_HD void flux_smooth_rev(const PointState<T>& st0, const Gas<T>& g, bool want_F, const T gF[5],
                             const T gdF[5], PointState<T>& cot) {
  const T* q = st0.q;
  const Prim<T> s = prim_of(q, g);
  const T H = g.h_r + q[4] + s.dp;
  T Qt[5];
  state_time_derivative(s, H, st0.dq, g, Qt);
  PrimBar<T> sb;
  prim_bar_zero(sb);
  T Hb = T(0);
  // dF = J_n(Q) Q_t, Q_t = -(J_0 dq_0 + J_1 dq_1 + J_2 dq_2)
  euler_jvp_rev_state<0>(s, H, Qt, g, gdF, sb, Hb);
  T Qtb[5] = {0, 0, 0, 0, 0};
  euler_jvp_rev_dq<0>(s, H, g, gdF, Qtb);
  T nQtb[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) nQtb[i] = -Qtb[i];
  euler_jvp_rev_state<0>(s, H, st0.dq[0], g, nQtb, sb, Hb);
  euler_jvp_rev_state<1>(s, H, st0.dq[1], g, nQtb, sb, Hb);
  euler_jvp_rev_state<2>(s, H, st0.dq[2], g, nQtb, sb, Hb);
  euler_jvp_rev_dq<0>(s, H, g, nQtb, cot.dq[0]);
  euler_jvp_rev_dq<1>(s, H, g, nQtb, cot.dq[1]);
  euler_jvp_rev_dq<2>(s, H, g, nQtb, cot.dq[2]);
  if (want_F) {
    // F = Euler flux + viscous flux (mu = viscosity(s), heat flux scaled by 1/Pr)
    euler_flux_dev_rev(s, q, g, gF, sb, cot.q);
    const T mu = viscosity(s, g);
    T mub = T(0);
    ns_viscous_flux_rev(s, st0.dq, g, mu, g.pr_fix + T(1), gF, sb, mub);
    if (g.visc_law == 1) sb.theta += mub * mu * g.visc_exp / s.theta;
    ns_viscous_vjp(s, g, mu, g.pr_fix + T(1), gF, cot.dq);
  }
  cot.q[4] += Hb;
  sb.dp += Hb;
  prim_of_rev(q, s, g, sb, cot.q);
}

// Cotangents of the values q and slopes dq of the equilibrium state of
// flux_full_eq as it enters the full flux (flux_full_combine): its three
// moment vectors V_k with the fit weights Fq[k] (F) and dFq[k] (dF), dual
// numbers carrying d/dtau, and the Prandtl fix -wpr tau p0 dT0 of F[4]
// (wpr = gF[4] pr_fix c_p), given the flux cotangents gF, gdF and the
// collision time tau; added to cot.  Returns the part's share of
// gF . dF/dtau + gdF . d(dF)/dtau.  The cotangents of mu0 and p0 through tau
// are applied by pressure_viscosity_rev.
template <class T>
HGKS_HD T flux_full_eq_rev(const PointState<T>& st0, const Gas<T>& g, const T gF[5], const T gdF[5],
                           const Dual<T> Fq[3], const Dual<T> dFq[3], T wpr, T tau, PointState<T>& cot) {
  const T* q = st0.q;
  const T* d0 = st0.dq[0];
  const Prim<T> s = prim_of(q, g);
  const T H = g.h_r + q[4] + s.dp;
  T Qt[5];
  state_time_derivative(s, H, st0.dq, g, Qt);
  // forward: V0 = Euler flux, V2 = J_n Q_t, V1 = -Fv(mu = p, Pr = 1) - V2, dT0
  T V0[5], V2[5], Fv[5];
  euler_flux_dev(s, q, g, V0);
  euler_jvp<0>(s, H, Qt, g, V2);
  ns_viscous_flux(s, st0.dq, g, s.p, T(1), Fv);
  const T q2 = s.U * s.U + s.V * s.V + s.W * s.W;
  const T dp0 = g.gm1 * (d0[4] - s.U * d0[1] - s.V * d0[2] - s.W * d0[3] + T(0.5) * q2 * d0[0]);
  const T dT = (dp0 - s.theta * d0[0]) * s.inv_rho;
  T phi = -wpr * s.p * dT;
  T gV0[5], Fvb[5], V2b[5];  // cotangents of V0, of Fv and of V2 (V1 = -Fv - V2)
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const T gt0 = gF[i] * Fq[0].d + gdF[i] * dFq[0].d, gt1 = gF[i] * Fq[1].d + gdF[i] * dFq[1].d;
    const T gt2 = gF[i] * Fq[2].d + gdF[i] * dFq[2].d;
    phi += gt0 * V0[i] + gt1 * (-Fv[i] - V2[i]) + gt2 * V2[i];
    const T gv1 = gF[i] * Fq[1].v + gdF[i] * dFq[1].v, gv2 = gF[i] * Fq[2].v + gdF[i] * dFq[2].v;
    gV0[i] = gF[i] * Fq[0].v + gdF[i] * dFq[0].v;
    Fvb[i] = -gv1;
    V2b[i] = gv2 - gv1;
  }
  // backward; the Prandtl fix gives p0 and dT0 the cotangents -wpr tau dT0
  // and -wpr tau p0
  const T gdT = -wpr * tau * s.p;
  PrimBar<T> sb;
  prim_bar_zero(sb);
  T Hb = T(0);
  {
    const T dp0b = gdT * s.inv_rho;
    sb.theta += -gdT * d0[0] * s.inv_rho;
    sb.inv += gdT * (dp0 - s.theta * d0[0]);
    sb.U += dp0b * g.gm1 * (s.U * d0[0] - d0[1]);
    sb.V += dp0b * g.gm1 * (s.V * d0[0] - d0[2]);
    sb.W += dp0b * g.gm1 * (s.W * d0[0] - d0[3]);
    temperature_slope_vjp(s, g, gdT, cot.dq[0]);
  }
  sb.p += -wpr * tau * dT;
  T mub = T(0);
  ns_viscous_flux_rev(s, st0.dq, g, s.p, T(1), Fvb, sb, mub);
  sb.p += mub;
  ns_viscous_vjp(s, g, s.p, T(1), Fvb, cot.dq);
  euler_jvp_rev_state<0>(s, H, Qt, g, V2b, sb, Hb);
  T Qtb[5] = {0, 0, 0, 0, 0};
  euler_jvp_rev_dq<0>(s, H, g, V2b, Qtb);
  // Q_t = -(J_0 dq_0 + J_1 dq_1 + J_2 dq_2)
  T nQtb[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) nQtb[i] = -Qtb[i];
  euler_jvp_rev_state<0>(s, H, st0.dq[0], g, nQtb, sb, Hb);
  euler_jvp_rev_state<1>(s, H, st0.dq[1], g, nQtb, sb, Hb);
  euler_jvp_rev_state<2>(s, H, st0.dq[2], g, nQtb, sb, Hb);
  euler_jvp_rev_dq<0>(s, H, g, nQtb, cot.dq[0]);
  euler_jvp_rev_dq<1>(s, H, g, nQtb, cot.dq[1]);
  euler_jvp_rev_dq<2>(s, H, g, nQtb, cot.dq[2]);
  euler_flux_dev_rev(s, q, g, gV0, sb, cot.q);
  // H = h_r + q4 + dp
  cot.q[4] += Hb;
  sb.dp += Hb;
  prim_of_rev(q, s, g, sb, cot.q);
  return phi;
}

// Adds to qb the cotangent of the values q through the pressure (gp) and the
// viscosity (gmu) of their state.
template <class T>
HGKS_HD void pressure_viscosity_rev(const T q[5], const Gas<T>& g, T gp, T gmu, T qb[5]) {
  const Prim<T> s = prim_of(q, g);
  PrimBar<T> sb;
  prim_bar_zero(sb);
  sb.p += gp;
  if (g.visc_law == 1) sb.theta += gmu * viscosity(s, g) * g.visc_exp / s.theta;
  prim_of_rev(q, s, g, sb, qb);
}

// Cotangents of the three states (st[0] = l, st[1] = r, st[2] = the
// compatibility state; values and slopes) of the full flux (flux_full) given
// the cotangents gF of F and gdF of dF; added to cot.  The fit weights
// Fq_k, dFq_k of Eq. (7) are formed as dual numbers in tau; each part runs
// one reverse pass with the cotangents gF Fq_k + gdF dFq_k of its moment
// vectors and returns its share of phi = gF . dF/dtau + gdF . d(dF)/dtau;
// phi then reaches the states through tau = mu0/p0 + C |p_l - p_r|/(p_l +
// p_r) dt.
template <class T>
HGKS_HD void flux_full_vjp(const PointState<T>* st, const Gas<T>& g, T dt, const T gF[5], const T gdF[5],
                           PointState<T>* cot) {
  T mu0, p0, pl, pr;
  {
    const Prim<T> s0 = prim_of(st[2].q, g);
    mu0 = viscosity(s0, g);
    p0 = s0.p;
    pl = prim_of(st[0].q, g).p;
    pr = prim_of(st[1].q, g).p;
  }
  const T tau = collision_time_full(mu0, p0, pl, pr, g, dt);
  Dual<T> Fq[6], dFq[6];
  fit_coefficients(Dual<T>(tau, T(1)), Dual<T>(dt), Fq, dFq);
  const T wpr = gF[4] * g.pr_fix * (T(0.5) * (g.K + T(5)));
  T phi = flux_full_eq_rev(st[2], g, gF, gdF, Fq, dFq, wpr, tau, cot[2]);
  // V_3 is the half-space sum minus the reference Euler flux (p_r in component 1).
  phi -= (gF[1] * Fq[3].d + gdF[1] * dFq[3].d) * g.p_r;
  // One copy of the half-space code for both sides: the side's state in and
  // its cotangent out through selects.
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const PointState<T> x = side == 0 ? st[0] : st[1];
    PointState<T> c;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      c.q[i] = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) c.dq[d][i] = T(0);
    }
    phi += flux_full_side_rev(x, g, side, gF, gdF, Fq + 3, dFq + 3, c);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (side == 0) cot[0].q[i] += c.q[i];
      else cot[1].q[i] += c.q[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (side == 0) cot[0].dq[d][i] += c.dq[d][i];
        else cot[1].dq[d][i] += c.dq[d][i];
      }
    }
  }
  const Gas<Dual<T>> gd = dual_gas(g);
  const T dtau_dpl =
      collision_time_full(Dual<T>(mu0), Dual<T>(p0), Dual<T>(pl, T(1)), Dual<T>(pr), gd, Dual<T>(dt)).d;
  const T dtau_dpr =
      collision_time_full(Dual<T>(mu0), Dual<T>(p0), Dual<T>(pl), Dual<T>(pr, T(1)), gd, Dual<T>(dt)).d;
  pressure_viscosity_rev(st[2].q, g, -phi * mu0 / (p0 * p0), phi / p0, cot[2].q);
  pressure_viscosity_rev(st[0].q, g, phi * dtau_dpl, T(0), cot[0].q);
  pressure_viscosity_rev(st[1].q, g, phi * dtau_dpr, T(0), cot[1].q);
}

}  // namespace hgks

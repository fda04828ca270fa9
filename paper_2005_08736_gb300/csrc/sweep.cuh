// Fused sweep kernel: for one direction d and one S2O4 stage, the face
// fields, the tangential reconstruction to the 2x2 Gauss points and the BGK
// flux there, for a 2D tile of faces marching along the normal.
//
// Tile: TP x TS faces in the transverse plane, P = the faster-varying
// transverse axis in memory, S = the slower one; the CTA marches through a
// chunk of faces f0..f1-1 along d (face f lies between cells f-1 and f).
// Per face layer:
//   phase 1  one thread per transverse point of the tile plus a halo of 2:
//            the six cells f-3..f+2 along d (L1-cached loads), WENO5 end
//            values of cells f-1 and f, the normal slopes, the compatibility
//            state Q0 and its normal slope -> face fields in shared memory;
//   phase 2  the tangential pass along t1 = d+1 for every point of the tile
//            (halo 2 along t2): values at the two t1 Gauss abscissae, and
//            t1-derivatives of the state fields -> shared memory;
//   phase 3  the tangential pass along t2 = d+2 and the flux at each Gauss
//            point; TPF threads per face, each with 4/TPF Gauss points,
//            summed with weights 1/4 into the face flux, written to HBM.
#pragma once

#include "charvars.cuh"
#include "compat.cuh"
#include "kernels.cuh"
#include "packed.cuh"

#include <type_traits>

namespace hgks {

template <class T>
struct SweepArgs {
  const T* __restrict__ q;     // padded state (deviation)
  T* __restrict__ fd;          // face fluxes [10][fbox]: F then dF, global frame
  const T* __restrict__ wn;    // widths along d (offset kGhost)
  const T* __restrict__ wt1;   // widths along t1
  const T* __restrict__ wt2;   // widths along t2
  const double* __restrict__ scal;
  GridDev g;
  int d;
  int chunk;
  int xt;  // d = x and q is the copy with x slowest ([5][x][z][y], k_transpose_x)
  Gas<T> gas;
};

template <int FLUX, int MODE = 0>
struct SweepLayout {
  static constexpr int NV = FLUX == FLUX_FULL ? 15 : 5;  // state field components
  static constexpr int QM = 2 * NV;                      // characteristic modes: Qm
  static constexpr int NFF = 2 * NV + (is_char_mode<MODE>() ? 5 : 0);  // + normal slopes (+ Qm)
  static constexpr int NT1 = 4 * NV + 2 * NV;            // t1 pass outputs
};

// Threads of a sweep CTA: 256, or one per face for tiles of more faces.
__host__ __device__ constexpr int sweep_threads(int tp, int ts) { return tp * ts > 256 ? tp * ts : 256; }

// Per-thread slots of the full-flux phase 3 with two threads per face: the
// three point states (20 values each) of the second t2 abscissa.
template <int FLUX, int TPF>
constexpr int sweep_scratch_elems() {
  return FLUX == FLUX_FULL && TPF == 2 ? 60 * 256 : 0;
}

template <class T, int MODE, int FLUX, int TP, int TS, int NL>
constexpr size_t sweep_smem_bytes() {
  constexpr int NH = (TP + 4) * (TS + 4);
  constexpr int TPF = sweep_threads(TP, TS) / (TP * TS);
  return sizeof(T) * ((NL * SweepLayout<FLUX, MODE>::NFF + SweepLayout<FLUX, MODE>::NT1) * NH +
                      (TPF - 1) * 10 * TP * TS + sweep_scratch_elems<FLUX, TPF>());
}

// Tangential reconstruction of a 5-vector field (components at src + i*sc,
// face averages at offsets -2..2 times sr): values v and derivatives d at the
// two Gauss abscissae, in the characteristic variables of b (the projection
// of every average, the scalar reconstruction per characteristic component,
// the map back).
template <int MODE, class T>
__device__ __forceinline__ void tangential_char(const T* src, int sc, int sr, const CharBasis<T>& b,
                                                T v[2][5], T d[2][5]) {
  T w[5][5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    T qv[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) qv[i] = src[i * sc + (r - 2) * sr];
    to_char(b, qv, w[r]);
  }
  T cv[2][5], cd[2][5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    T vv[2], dd[2];
    tangential<MODE>(w[0][i], w[1][i], w[2][i], w[3][i], w[4][i], vv, dd);
    cv[0][i] = vv[0];
    cv[1][i] = vv[1];
    cd[0][i] = dd[0];
    cd[1][i] = dd[1];
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    from_char(b, cv[m], v[m]);
    from_char(b, cd[m], d[m]);
  }
}

// t2 pass of the state group s (fields 5s..5s+4 of the t1-pass output) at t1
// abscissa m1 for the face at at3: value, t2-derivative (per cell length),
// t1-derivative field and normal-slope field at both t2 abscissae.
template <class T, int MODE, int NV, int NH>
__device__ __forceinline__ void t2_group(const T* tb, int s, int m1, int at3, int st2,
                                         const CharBasis<T>& b, T val[2][5], T dt2[2][5],
                                         T dt1[2][5], T dn[2][5]) {
  const T* sv = tb + (4 * (5 * s) + m1) * NH + at3;
  const T* sdv = tb + (4 * (5 * s) + 2 + m1) * NH + at3;
  const T* ss = tb + (4 * NV + 2 * (5 * s) + m1) * NH + at3;
  if constexpr (is_char_mode<MODE>()) {
    T scratch[2][5];
    tangential_char<MODE>(sv, 4 * NH, st2, b, val, dt2);
    tangential_char<MODE>(sdv, 4 * NH, st2, b, dt1, scratch);
    tangential_char<MODE>(ss, 2 * NH, st2, b, dn, scratch);
  } else {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T* a = sv + 4 * i * NH;
      const T* c = sdv + 4 * i * NH;
      const T* e = ss + 2 * i * NH;
      T v[2], dd[2], vd[2], vs[2];
      tangential<MODE>(a[-2 * st2], a[-st2], a[0], a[st2], a[2 * st2], v, dd);
      tangential_val<MODE>(c[-2 * st2], c[-st2], c[0], c[st2], c[2 * st2], vd);
      tangential_val<MODE>(e[-2 * st2], e[-st2], e[0], e[st2], e[2 * st2], vs);
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        val[m][i] = v[m];
        dt2[m][i] = dd[m];
        dt1[m][i] = vd[m];
        dn[m][i] = vs[m];
      }
    }
  }
}

// Geometry of one sweep: normal axis d, transverse axes P (faster in memory)
// and S, and the first tangential axis t1 = d+1.
struct SweepAxes {
  int d, P, S;
  bool t1P;        // t1 is P (d = x, z) or S (d = y)
  long long sd;    // stride of the padded state along d
  int gv[5];       // global variable of each local-frame component
  bool xt;         // the state is the copy with x slowest (x sweep)
  // Padded index of cell (x, y, z) in the state the sweep reads.
  __device__ __forceinline__ long long index(const GridDev& g, int x, int y, int z) const {
    return xt ? ((long long)(x + kGhost) * g.p[2] + (z + kGhost)) * g.p[1] + (y + kGhost)
              : pad_index(g, x, y, z);
  }
};
__device__ __forceinline__ SweepAxes sweep_axes(int d, const GridDev& g, bool xt = false) {
  SweepAxes a;
  a.d = d;
  a.P = d == 0 ? 1 : 0;
  a.S = d == 2 ? 1 : 2;
  a.t1P = ((d + 1) % 3) == a.P;
  a.xt = xt && d == 0;
  a.sd = a.xt ? (long long)g.p[1] * g.p[2]
              : (d == 0 ? 1LL : (d == 1 ? (long long)g.p[0] : (long long)g.p[0] * g.p[1]));
#pragma unroll
  for (int i = 0; i < 5; ++i) a.gv[i] = global_var(d, i);
  return a;
}

// Face fields (conservative-variable reconstruction) of one face point from
// the six cells f-3..f+2 along the normal, qa[i][k] = variable i of cell
// f-3+k (local frame), and the widths hl, hr of cells f-1 and f: the WENO5
// end values, the normal slopes, the compatibility state Q0 and its normal
// slope, into ff[k * NH + h].
template <class T, int MODE, int FLUX, int NH>
HGKS_HD void face_fields_cells(const T qa[5][6], T hl, T hr, const Gas<T>& gas,
                                                  int h, T* ff) {
  const T rhl = T(1) / hl, rhr = T(1) / hr, r6 = T(1) / (T(6) * (hl + hr));
  T Ql[5], Qr[5], Dl[5], Dr[5], D0[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const T q0 = qa[i][0], q1 = qa[i][1], q2 = qa[i][2], q3 = qa[i][3], q4 = qa[i][4], q5 = qa[i][5];
    T Li, Ri, Lr, Rr;
    bool packed = false;
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<T, float>::value && recon_of<MODE>() != RECON_LINEAR) {
      // Both cells' WENO5 pairs in the halves of packed FP32 pairs.
      float2 L2, R2;
      weno5_pair_x2<recon_of<MODE>()>(make_float2(q0, q1), make_float2(q1, q2), make_float2(q2, q3),
                                      make_float2(q3, q4), make_float2(q4, q5), L2, R2);
      Li = L2.x;
      Ri = R2.x;
      Lr = L2.y;
      Rr = R2.y;
      packed = true;
    }
#endif
    if (!packed) {
      weno5_pair<MODE>(q0, q1, q2, q3, q4, Li, Ri);
      weno5_pair<MODE>(q1, q2, q3, q4, q5, Lr, Rr);
    }
    Ql[i] = Ri;
    Qr[i] = Lr;
    Dl[i] = (T(4) * Ri + T(2) * Li - T(6) * q2) * rhl;
    Dr[i] = -(T(4) * Lr + T(2) * Rr - T(6) * q3) * rhr;
    D0[i] = (q1 - T(15) * q2 + T(15) * q3 - q4) * r6;
  }
  T Q0[5];
  compat_state(Ql, Qr, gas, Q0);
  if constexpr (FLUX == FLUX_SMOOTH) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      ff[i * NH + h] = Q0[i];
      ff[(5 + i) * NH + h] = D0[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      ff[i * NH + h] = Ql[i];
      ff[(5 + i) * NH + h] = Qr[i];
      ff[(10 + i) * NH + h] = Q0[i];
      ff[(15 + i) * NH + h] = Dl[i];
      ff[(20 + i) * NH + h] = Dr[i];
      ff[(25 + i) * NH + h] = D0[i];
    }
  }
}

// Face fields of the x sweep (conservative variables) for the layers
// fb .. fb+nl-1 at transverse point (Pc, Sc): one thread reads the nl+5 cells
// fb-3 .. fb+nl+1 along x of each variable, contiguous in memory, as pairs
// (two-element vector loads; the caller guarantees an even padded row length,
// so that with fb even every pair is aligned), and forms the fields of each
// layer l into ffb + l * NFF * NH.
template <class T, int MODE, int FLUX, int NH, int NL, int NFF>
__device__ __forceinline__ void face_fields_x_item(const T* __restrict__ q, const GridDev& g,
                                                   const SweepAxes& ax, const T* __restrict__ wn,
                                                   const Gas<T>& gas, int fb, int nl, int Pc, int Sc,
                                                   int h, T* ffb) {
  using V2 = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
  constexpr int NC = NL + 5;  // cells of NL layers
  const long long cb = pad_index(g, fb - 3, ax.P == 1 ? Pc : Sc, ax.P == 1 ? Sc : Pc);
  T cells[5][NC + 1];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const T* qv = q + ax.gv[i] * g.P + cb;
#pragma unroll
    for (int j = 0; j < (NC + 1) / 2; ++j) {
      if (2 * j + 1 < nl + 5) {
        const V2 v = __ldg(reinterpret_cast<const V2*>(qv + 2 * j));
        cells[i][2 * j] = v.x;
        cells[i][2 * j + 1] = v.y;
      } else if (2 * j < nl + 5) {
        cells[i][2 * j] = __ldg(qv + 2 * j);
        cells[i][2 * j + 1] = T(0);
      } else {
        cells[i][2 * j] = cells[i][2 * j + 1] = T(0);
      }
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (l < nl) {
      T qa[5][6];
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int k = 0; k < 6; ++k) qa[i][k] = cells[i][l + k];
      const int f = fb + l;
      face_fields_cells<T, MODE, FLUX, NH>(qa, wn[f - 1 + kGhost], wn[f + kGhost], gas, h,
                                           ffb + l * NFF * NH);
    }
  }
}

// Face fields of face layer f at transverse point (Pc, Sc) into ff[k * NH + h]:
// WENO5 end values of cells f-1 and f, their normal slopes, the compatibility
// state Q0 and its normal slope (local frame).  Smooth flux: fields Q0, dQ0/dn;
// full flux: Q_l, Q_r, Q0, dQ_l/dn, dQ_r/dn, dQ0/dn.
template <class T, int MODE, int FLUX, int NH>
__device__ __forceinline__ void face_fields_item(const T* __restrict__ q, const GridDev& g,
                                                 const SweepAxes& ax, const T* __restrict__ wn,
                                                 const Gas<T>& gas, int f, int Pc, int Sc, int h,
                                                 T* ff) {
  int c[3];
  c[ax.d] = f - 3;
  c[ax.P] = Pc;
  c[ax.S] = Sc;
  const long long cb = ax.index(g, c[0], c[1], c[2]);
  const long long sd = ax.sd;
  const T hl = wn[f - 1 + kGhost], hr = wn[f + kGhost];
  if constexpr (!is_char_mode<MODE>()) {
    T qa[5][6];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T* qv = q + ax.gv[i] * g.P + cb;
#pragma unroll
      for (int k = 0; k < 6; ++k) qa[i][k] = __ldg(qv + k * sd);
    }
    face_fields_cells<T, MODE, FLUX, NH>(qa, hl, hr, gas, h, ff);
  } else {
    // Characteristic variables of Qm, the mean of the two cells beside the face.
    const T rhl = T(1) / hl, rhr = T(1) / hr, r6 = T(1) / (T(6) * (hl + hr));
    T Ql[5], Qr[5], Dl[5], Dr[5], D0[5];
    T qa[6][5], qm[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T* qv = q + ax.gv[i] * g.P + cb;
#pragma unroll
      for (int k = 0; k < 6; ++k) qa[k][i] = __ldg(qv + k * sd);
      qm[i] = T(0.5) * (qa[2][i] + qa[3][i]);
    }
    const CharBasis<T> b = char_basis(qm, gas);
    T w[6][5];
#pragma unroll
    for (int k = 0; k < 6; ++k) to_char(b, qa[k], w[k]);
    T e[4][5];  // Q at x_{i+1/2} and x_{i-1/2} from cell i, at x_{i+1/2} and x_{i+3/2} from cell i+1
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      weno5_pair<MODE>(w[0][i], w[1][i], w[2][i], w[3][i], w[4][i], e[1][i], e[0][i]);
      weno5_pair<MODE>(w[1][i], w[2][i], w[3][i], w[4][i], w[5][i], e[2][i], e[3][i]);
    }
    T E[4][5];
#pragma unroll
    for (int k = 0; k < 4; ++k) from_char(b, e[k], E[k]);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      Ql[i] = E[0][i];
      Qr[i] = E[2][i];
      Dl[i] = (T(4) * E[0][i] + T(2) * E[1][i] - T(6) * qa[2][i]) * rhl;
      Dr[i] = -(T(4) * E[2][i] + T(2) * E[3][i] - T(6) * qa[3][i]) * rhr;
      D0[i] = (qa[1][i] - T(15) * qa[2][i] + T(15) * qa[3][i] - qa[4][i]) * r6;
      ff[(SweepLayout<FLUX, MODE>::QM + i) * NH + h] = qm[i];
    }
    T Q0[5];
    compat_state(Ql, Qr, gas, Q0);
    if constexpr (FLUX == FLUX_SMOOTH) {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        ff[i * NH + h] = Q0[i];
        ff[(5 + i) * NH + h] = D0[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        ff[i * NH + h] = Ql[i];
        ff[(5 + i) * NH + h] = Qr[i];
        ff[(10 + i) * NH + h] = Q0[i];
        ff[(15 + i) * NH + h] = Dl[i];
        ff[(20 + i) * NH + h] = Dr[i];
        ff[(25 + i) * NH + h] = D0[i];
      }
    }
  }
}

// Tangential pass along t1 for one point `at` of the tile (stride st1 in the
// shared-memory plane): values at both t1 Gauss abscissae of every field and
// t1-derivatives of the state fields, into tb.
template <class T, int MODE, int FLUX, int NH>
__device__ __forceinline__ void t1_pass_item(const T* ff, T* tb, int at, int st1, const Gas<T>& gas) {
  constexpr int NV = SweepLayout<FLUX>::NV;
  if constexpr (is_char_mode<MODE>()) {
    // Characteristic variables of Qm at the centre point.
    T qm[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) qm[i] = ff[(SweepLayout<FLUX, MODE>::QM + i) * NH + at];
    const CharBasis<T> b = char_basis(qm, gas);
#pragma unroll 1
    for (int grp = 0; grp < 2 * NV / 5; ++grp) {
      // groups 0 .. NV/5-1: state fields (values and t1-derivatives);
      // then their normal slopes (values only)
      const bool state = grp < NV / 5;
      const int k0 = 5 * grp;  // first field of the group in ff
      T v[2][5], d[2][5];
      tangential_char<MODE>(ff + k0 * NH + at, NH, st1, b, v, d);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        if (state) {
          const int k = k0 + i;
          tb[(4 * k + 0) * NH + at] = v[0][i];
          tb[(4 * k + 1) * NH + at] = v[1][i];
          tb[(4 * k + 2) * NH + at] = d[0][i];
          tb[(4 * k + 3) * NH + at] = d[1][i];
        } else {
          const int k = k0 - NV + i;
          tb[(4 * NV + 2 * k + 0) * NH + at] = v[0][i];
          tb[(4 * NV + 2 * k + 1) * NH + at] = v[1][i];
        }
      }
    }
  } else {
#pragma unroll(FLUX == FLUX_SMOOTH ? 5 : 1)
  for (int k = 0; k < NV; ++k) {
    const T* src = ff + k * NH + at;
    T v[2], dd[2];
    tangential<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v, dd);
    tb[(4 * k + 0) * NH + at] = v[0];
    tb[(4 * k + 1) * NH + at] = v[1];
    tb[(4 * k + 2) * NH + at] = dd[0];
    tb[(4 * k + 3) * NH + at] = dd[1];
  }
#pragma unroll(FLUX == FLUX_SMOOTH ? 5 : 1)
  for (int k = 0; k < NV; ++k) {
    const T* src = ff + (NV + k) * NH + at;
    T v[2];
    tangential_val<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v);
    tb[(4 * NV + 2 * k + 0) * NH + at] = v[0];
    tb[(4 * NV + 2 * k + 1) * NH + at] = v[1];
  }
  }
}

// One group of five fields of the t1 pass at point `at`: group g < NV/5 is
// state group g (values at both t1 abscissae and t1-derivatives), else the
// normal slopes of state group g - NV/5 (values only).
template <class T, int MODE, int NV, int NH>
HGKS_HD void t1_pass_group(const T* ff, T* tb, int at, int st1, int grp) {
  if (grp < NV / 5) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int k = 5 * grp + i;
      const T* src = ff + k * NH + at;
      T v[2], dd[2];
      tangential<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v, dd);
      tb[(4 * k + 0) * NH + at] = v[0];
      tb[(4 * k + 1) * NH + at] = v[1];
      tb[(4 * k + 2) * NH + at] = dd[0];
      tb[(4 * k + 3) * NH + at] = dd[1];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int j = 5 * (grp - NV / 5) + i;  // state field whose normal slope this is
      const T* src = ff + (NV + j) * NH + at;
      T v[2];
      tangential_val<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v);
      tb[(4 * NV + 2 * j + 0) * NH + at] = v[0];
      tb[(4 * NV + 2 * j + 1) * NH + at] = v[1];
    }
  }
}

// t1_pass_group in FP32 with nonlinear weights: the five fields of the
// group two at a time in packed FP32 pairs (fields 0 and 1, 2 and 3), the
// fifth alone; the same outputs and layout.
template <int MODE, int NV, int NH>
__device__ __forceinline__ void t1_pass_group_wx2(const float* ff, float* tb, int at, int st1, int grp) {
  const bool state = grp < NV / 5;
  // first field of the group in ff
  const int kf = state ? 5 * grp : NV + 5 * (grp - NV / 5);
#pragma unroll
  for (int i = 0; i < 4; i += 2) {
    const float* sa = ff + (kf + i) * NH + at;
    const float* sb = sa + NH;
    float2 f[5], v[2], dd[2];
#pragma unroll
    for (int j = 0; j < 5; ++j) f[j] = make_float2(sa[(j - 2) * st1], sb[(j - 2) * st1]);
    tangential_weno_x2<MODE>(f[0], f[1], f[2], f[3], f[4], v, dd);
    if (state) {
      const int k = kf + i;
      tb[(4 * k + 0) * NH + at] = v[0].x;
      tb[(4 * k + 1) * NH + at] = v[1].x;
      tb[(4 * k + 2) * NH + at] = dd[0].x;
      tb[(4 * k + 3) * NH + at] = dd[1].x;
      tb[(4 * k + 4) * NH + at] = v[0].y;
      tb[(4 * k + 5) * NH + at] = v[1].y;
      tb[(4 * k + 6) * NH + at] = dd[0].y;
      tb[(4 * k + 7) * NH + at] = dd[1].y;
    } else {
      const int j = kf - NV + i;  // state field whose normal slope this is
      tb[(4 * NV + 2 * j + 0) * NH + at] = v[0].x;
      tb[(4 * NV + 2 * j + 1) * NH + at] = v[1].x;
      tb[(4 * NV + 2 * j + 2) * NH + at] = v[0].y;
      tb[(4 * NV + 2 * j + 3) * NH + at] = v[1].y;
    }
  }
  {
    const float* src = ff + (kf + 4) * NH + at;
    float v[2], dd[2];
    tangential<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v, dd);
    if (state) {
      const int k = kf + 4;
      tb[(4 * k + 0) * NH + at] = v[0];
      tb[(4 * k + 1) * NH + at] = v[1];
      tb[(4 * k + 2) * NH + at] = dd[0];
      tb[(4 * k + 3) * NH + at] = dd[1];
    } else {
      const int j = kf - NV + 4;
      tb[(4 * NV + 2 * j + 0) * NH + at] = v[0];
      tb[(4 * NV + 2 * j + 1) * NH + at] = v[1];
    }
  }
}

// t1_pass_group with the packed layout of the last phase (FP32, linear
// weights): the outputs at the two t1 abscissae are stored side by side as a
// float2 -- state field k: pair plane 2k (values), 2k+1 (t1-derivatives);
// normal slope of state field j: pair plane 2 NV + j (values).
template <int MODE, int NV, int NH>
__device__ __forceinline__ void t1_pass_group_x2(const float* ff, float* tb, int at, int st1, int grp) {
  float2* tb2 = reinterpret_cast<float2*>(tb);
  if (grp < NV / 5) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int k = 5 * grp + i;
      const float* src = ff + k * NH + at;
      float v[2], dd[2];
      tangential<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v, dd);
      tb2[(2 * k) * NH + at] = make_float2(v[0], v[1]);
      tb2[(2 * k + 1) * NH + at] = make_float2(dd[0], dd[1]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int j = 5 * (grp - NV / 5) + i;
      const float* src = ff + (NV + j) * NH + at;
      float v[2];
      tangential_val<MODE>(src[-2 * st1], src[-st1], src[0], src[st1], src[2 * st1], v);
      tb2[(2 * NV + j) * NH + at] = make_float2(v[0], v[1]);
    }
  }
}

// Resident CTAs per SM the register budget is sized for: the smooth FP32
// sweep fits three (shared memory allows three as well), the others one or two
// (two at most for the characteristic modes, which need more registers).
template <class T, int FLUX> struct SweepOccupancy { static constexpr int value = 1; };
template <> struct SweepOccupancy<float, FLUX_SMOOTH> { static constexpr int value = 3; };
template <> struct SweepOccupancy<double, FLUX_SMOOTH> { static constexpr int value = 2; };

// Resident CTAs per SM for the register budget: SweepOccupancy for 256
// threads (two at most in the characteristic modes); tiles of 384 threads
// two, of 512 one.
template <class T, int MODE, int FLUX, int TP, int TS>
__host__ __device__ constexpr int sweep_min_blocks() {
  return sweep_threads(TP, TS) == 512   ? 1
         : sweep_threads(TP, TS) == 384 ? 2
         : is_char_mode<MODE>() && SweepOccupancy<T, FLUX>::value > 2 ? 2
                                                                      : SweepOccupancy<T, FLUX>::value;
}

// PK (FP32, linear weights, smooth flux, one thread per face): the last
// phase evaluates the two t1 abscissae of a face as the halves of packed FP32
// pairs (packed.cuh); shared memory allows two CTAs per SM for this tile, so
// the register budget is sized for two.
template <class T, int MODE, int FLUX, int STAGE, int TP, int TS, int NL, bool PK = false>
__global__ void __launch_bounds__(sweep_threads(TP, TS), (PK ? 2 : sweep_min_blocks<T, MODE, FLUX, TP, TS>()))
    k_sweep(SweepArgs<T> a) {
#define HGKS_SW_BX blockIdx.x
#define HGKS_SW_BY blockIdx.y
#define HGKS_SW_BZ blockIdx.z
#include "sweep_body.inc"
#undef HGKS_SW_BX
#undef HGKS_SW_BY
#undef HGKS_SW_BZ
}

}  // namespace hgks

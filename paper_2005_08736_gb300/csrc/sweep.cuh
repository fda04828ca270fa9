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
    weno5_pair<MODE>(q0, q1, q2, q3, q4, Li, Ri);
    weno5_pair<MODE>(q1, q2, q3, q4, q5, Lr, Rr);
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
  constexpr int HP = TP + 4, HS = TS + 4, NH = HP * HS;
  constexpr int NV = SweepLayout<FLUX>::NV;
  constexpr int NFF = SweepLayout<FLUX, MODE>::NFF;
  constexpr int NFACE = TP * TS;
  constexpr int NT = sweep_threads(TP, TS);  // threads of the CTA
  constexpr int TPF = NT / NFACE;  // threads per face in phase 3
  constexpr int GPF = 4 / TPF;      // Gauss points per thread
  static_assert(TPF * NFACE == NT && GPF * TPF == 4, "tile must give 1, 2 or 4 threads per face");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ffb = reinterpret_cast<T*>(smem_raw);  // [NL][NFF][NH]
  T* tb = ffb + NL * NFF * NH;              // [NT1][NH]
  T* part = tb + SweepLayout<FLUX>::NT1 * NH;  // [TPF-1][10][NFACE]
  T* scr = part + (TPF - 1) * 10 * NFACE;      // [60][256] (full flux, TPF = 2)

  const int d = a.d;
  const SweepAxes ax = sweep_axes(d, a.g, a.xt != 0);
  const int P = ax.P, S = ax.S;
  const bool t1P = ax.t1P;
  const int nP = a.g.n[P], nS = a.g.n[S], nd = a.g.n[d];
  const int p0 = blockIdx.x * TP, s0 = blockIdx.y * TS;
  const int f0 = blockIdx.z * a.chunk;
  const int f1 = min(f0 + a.chunk, nd + 1);
  const int tid = threadIdx.x;

  // Phase-3 role: one face and GPF Gauss points of it.
  const int face = tid % NFACE, sub = tid / NFACE;
  const int ip = face % TP, is = face / TP;
  const bool f_valid = (p0 + ip < nP) && (s0 + is < nS);
  const int cP = min(p0 + ip, nP - 1), cS = min(s0 + is, nS - 1);
  const int ct1 = t1P ? cP : cS, ct2 = t1P ? cS : cP;
  const T rh1 = T(1) / a.wt1[ct1 + kGhost], rh2 = T(1) / a.wt2[ct2 + kGhost];
  const int at3 = (is + 2) * HP + (ip + 2);
  const int st2 = t1P ? HP : 1;
  const T dt = T(a.scal[0]);
  const long long FS = (long long)(a.g.n[0] + (d == 0)) * (a.g.n[1] + (d == 1)) * (a.g.n[2] + (d == 2));
  // Face-flux layout: x fastest for the y and z faces; y fastest ([z][x][y])
  // for the x faces, so that the tile's threads (running along y) store
  // contiguously; the update kernel reads them through a shared-memory transpose.
  long long fout, fstep;
  if (d == 0) {
    fout = (long long)cS * (a.g.n[0] + 1) * a.g.n[1] + cP;
    fstep = a.g.n[1];
  } else {
    int c[3];
    c[d] = 0;
    c[P] = cP;
    c[S] = cS;
    fout = ((long long)c[2] * (a.g.n[1] + (d == 1)) + c[1]) * (a.g.n[0] + (d == 0)) + c[0];
    fstep = d == 1 ? (long long)a.g.n[0] : (long long)a.g.n[0] * a.g.n[1];
  }

  for (int fb = f0; fb < f1; fb += NL) {
    // ---------------- phase 1: face fields of layers fb .. fb+NL-1 ----------------
    // Items (layer, transverse point of the tile plus a halo of 2).  For d = x
    // consecutive threads take consecutive layers, so that the loads along x
    // are coalesced; otherwise consecutive transverse points along P (= x).
    if (NL == 2 && !is_char_mode<MODE>() && d == 0 && !ax.xt && (a.g.p[0] & 1) == 0) {
      // x sweep: one item per transverse point for both layers (pair loads
      // along x; fb is even because chunks and NL are).  Tiles with more
      // layers per pass keep the per-layer items below (register budget).
      const int nl = min(NL, f1 - fb);
      for (int h = tid; h < NH; h += NT) {
        const int hp = h % HP, hs = h / HP;
        const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
        if (Pc <= nP + 1 && Sc <= nS + 1) {
          face_fields_x_item<T, MODE, FLUX, NH, NL, NFF>(a.q, a.g, ax, a.wn, a.gas, fb, nl, Pc, Sc, h, ffb);
        } else {
#pragma unroll 1
          for (int l = 0; l < NL; ++l)
#pragma unroll 1
            for (int k = 0; k < NFF; ++k) ffb[(l * NFF + k) * NH + h] = T(0);
        }
#pragma unroll 1
        for (int l = nl; l < NL; ++l)
#pragma unroll 1
          for (int k = 0; k < NFF; ++k) ffb[(l * NFF + k) * NH + h] = T(0);
      }
    } else if (PK && !(d == 0 && !ax.xt)) {
      if constexpr (PK) {
        // Packed variant: one item per pair of adjacent points along P (the
        // state is contiguous along P, so both points' cells are neighbours);
        // pairs that reach past the grid's halo take the per-point path.
        static_assert(HP % 2 == 0, "point pairs must not straddle a row");
        constexpr int NH2 = NH / 2;
        for (int it = tid; it < NL * NH2; it += NT) {
          const int l = it / NH2, h = 2 * (it % NH2);
          const int f = fb + l;
          const int hp = h % HP, hs = h / HP;
          const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
          T* ff = ffb + l * NFF * NH;
          const bool ok0 = f < f1 && Pc <= nP + 1 && Sc <= nS + 1;
          const bool ok1 = ok0 && Pc + 1 <= nP + 1;
          if (ok1) {
            // Cell f-3 along d at (Pc, Sc): P = y, S = z for d = x; P = x otherwise.
            const int cx = d == 0 ? f - 3 : Pc;
            const int cy = d == 0 ? Pc : (d == 1 ? f - 3 : Sc);
            const int cz = d == 2 ? f - 3 : Sc;
            const long long cb = ax.index(a.g, cx, cy, cz);
            float2 qk[5][6];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              const T* qv = a.q + ax.gv[i] * a.g.P + cb;
#pragma unroll
              for (int k = 0; k < 6; ++k) qk[i][k] = make_float2(__ldg(qv + k * ax.sd), __ldg(qv + k * ax.sd + 1));
            }
            float2 Q0[5], D0[5];
            face_fields_smooth_linear_x2(qk, a.wn[f - 1 + kGhost], a.wn[f + kGhost], a.gas, Q0, D0);
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              *reinterpret_cast<float2*>(ff + i * NH + h) = Q0[i];
              *reinterpret_cast<float2*>(ff + (5 + i) * NH + h) = D0[i];
            }
          } else {
#pragma unroll 1
            for (int e2 = 0; e2 < 2; ++e2) {
              const bool ok = e2 == 0 ? ok0 : (f < f1 && Pc + 1 <= nP + 1 && Sc <= nS + 1);
              if (ok) {
                face_fields_item<T, MODE, FLUX, NH>(a.q, a.g, ax, a.wn, a.gas, f, Pc + e2, Sc, h + e2, ff);
              } else {
#pragma unroll 1
                for (int k = 0; k < NFF; ++k) ff[k * NH + h + e2] = T(0);
              }
            }
          }
        }
      }
    } else
    for (int it = tid; it < NL * NH; it += NT) {
      // Consecutive threads: consecutive layers for the x sweep reading q
      // (cells along x are contiguous), else consecutive points along P.
      const bool by_layer = d == 0 && !ax.xt;
      const int l = by_layer ? it % NL : it / NH;
      const int h = by_layer ? it / NL : it % NH;
      const int f = fb + l;
      const int hp = h % HP, hs = h / HP;
      const int Pc = p0 - 2 + hp, Sc = s0 - 2 + hs;
      T* ff = ffb + l * NFF * NH;
      if (f < f1 && Pc <= nP + 1 && Sc <= nS + 1) {
        face_fields_item<T, MODE, FLUX, NH>(a.q, a.g, ax, a.wn, a.gas, f, Pc, Sc, h, ff);
      } else {
#pragma unroll 1
        for (int k = 0; k < NFF; ++k) ff[k * NH + h] = T(0);
      }
    }
    __syncthreads();

#pragma unroll 1
  for (int l = 0; l < NL && fb + l < f1; ++l) {
    const int f = fb + l;
    const T* ff = ffb + l * NFF * NH;
    // ---------------- phase 2: tangential pass along t1 ----------------
    // Points of the tile with a halo of 2 along t2.  Conservative variables:
    // the (group of five fields, point) pairs are spread evenly over the CTA;
    // characteristic variables: one point (all fields) per item.
    if constexpr (is_char_mode<MODE>()) {
      const int items = t1P ? TP * HS : HP * TS;
      const int st1 = t1P ? 1 : HP;
      for (int it = tid; it < items; it += NT) {
        const int hp2 = t1P ? 2 + it % TP : it % HP;
        const int hs2 = t1P ? it / TP : 2 + it / HP;
        t1_pass_item<T, MODE, FLUX, NH>(ff, tb, hs2 * HP + hp2, st1, a.gas);
      }
    } else if (t1P) {
      constexpr int ITEMS = TP * HS;
#pragma unroll 1
      for (int it = tid; it < ITEMS * 2 * NV / 5; it += NT) {
        const int grp = it / ITEMS, pt = it % ITEMS;
        if constexpr (PK) t1_pass_group_x2<MODE, NV, NH>(ff, tb, (pt / TP) * HP + 2 + pt % TP, 1, grp);
        else t1_pass_group<T, MODE, NV, NH>(ff, tb, (pt / TP) * HP + 2 + pt % TP, 1, grp);
      }
    } else {
      constexpr int ITEMS = HP * TS;
#pragma unroll 1
      for (int it = tid; it < ITEMS * 2 * NV / 5; it += NT) {
        const int grp = it / ITEMS, pt = it % ITEMS;
        if constexpr (PK) t1_pass_group_x2<MODE, NV, NH>(ff, tb, (2 + pt / HP) * HP + pt % HP, HP, grp);
        else t1_pass_group<T, MODE, NV, NH>(ff, tb, (2 + pt / HP) * HP + pt % HP, HP, grp);
      }
    }
    __syncthreads();

    // ---------------- phase 3: tangential pass along t2 and flux ----------------
    // Characteristic modes: the basis of Qm at this thread's face.
    CharBasis<T> cbs{};
    if constexpr (is_char_mode<MODE>()) {
      T qm[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) qm[i] = ff[(SweepLayout<FLUX, MODE>::QM + i) * NH + at3];
      cbs = char_basis(qm, a.gas);
    }
    T Fs[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) Fs[i] = T(0);
    if constexpr (PK) {
      // Both t1 abscissae at once, as the halves of packed pairs: one pass
      // along t2 per field gives both t2 abscissae; the flux at (., m2) is
      // evaluated for the two t1 abscissae together.
      static_assert(std::is_same<T, float>::value && MODE == RECON_LINEAR && FLUX == FLUX_SMOOTH &&
                        TPF == 1, "packed phase 3: FP32, linear weights, smooth flux, one thread per face");
      const float2* tb2 = reinterpret_cast<const float2*>(tb);
      PointStateX2 st[2];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const float2* sv = tb2 + (2 * i) * NH + at3;
        const float2* sdv = tb2 + (2 * i + 1) * NH + at3;
        const float2* ss = tb2 + (2 * NV + i) * NH + at3;
        float2 v[2], dd[2], vd[2], vs[2];
        tangential_linear_x2(sv[-2 * st2], sv[-st2], sv[0], sv[st2], sv[2 * st2], v, dd);
        tangential_linear_val_x2(sdv[-2 * st2], sdv[-st2], sdv[0], sdv[st2], sdv[2 * st2], vd);
        tangential_linear_val_x2(ss[-2 * st2], ss[-st2], ss[0], ss[st2], ss[2 * st2], vs);
#pragma unroll
        for (int m2 = 0; m2 < 2; ++m2) {
          st[m2].q[i] = v[m2];
          st[m2].dq[0][i] = vs[m2];
          st[m2].dq[1][i] = mul2(vd[m2], bc2(rh1));
          st[m2].dq[2][i] = mul2(dd[m2], bc2(rh2));
        }
      }
      flux_smooth_x2<STAGE == 1>(st[0], a.gas, Fs);
      flux_smooth_x2<STAGE == 1>(st[1], a.gas, Fs);
    } else if constexpr (FLUX == FLUX_SMOOTH && TPF <= 2) {
      // One pass along t2 gives both t2 abscissae: each thread takes one (or
      // both) t1 abscissae m1 and evaluates the flux at (m1, 0) and (m1, 1).
#pragma unroll 1
      for (int m1 = (TPF == 2 ? sub : 0); m1 < (TPF == 2 ? sub + 1 : 2); ++m1) {
        PointState<T> st[2];
        if constexpr (is_char_mode<MODE>()) {
          T val[2][5], d2[2][5], d1[2][5], dn[2][5];
          t2_group<T, MODE, NV, NH>(tb, 0, m1, at3, st2, cbs, val, d2, d1, dn);
#pragma unroll
          for (int m2 = 0; m2 < 2; ++m2)
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              st[m2].q[i] = val[m2][i];
              st[m2].dq[0][i] = dn[m2][i];
              st[m2].dq[1][i] = d1[m2][i] * rh1;
              st[m2].dq[2][i] = d2[m2][i] * rh2;
            }
        } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          const T* sv = tb + (4 * i + m1) * NH + at3;
          const T* sdv = tb + (4 * i + 2 + m1) * NH + at3;
          const T* ss = tb + (4 * NV + 2 * i + m1) * NH + at3;
          T v[2], dd[2], vd[2], vs[2];
          tangential<MODE>(sv[-2 * st2], sv[-st2], sv[0], sv[st2], sv[2 * st2], v, dd);
          tangential_val<MODE>(sdv[-2 * st2], sdv[-st2], sdv[0], sdv[st2], sdv[2 * st2], vd);
          tangential_val<MODE>(ss[-2 * st2], ss[-st2], ss[0], ss[st2], ss[2 * st2], vs);
#pragma unroll
          for (int m2 = 0; m2 < 2; ++m2) {
            st[m2].q[i] = v[m2];
            st[m2].dq[0][i] = vs[m2];
            st[m2].dq[1][i] = vd[m2] * rh1;
            st[m2].dq[2][i] = dd[m2] * rh2;
          }
        }
        }
#pragma unroll
        for (int m2 = 0; m2 < 2; ++m2) {
          T F[5], dF[5];
          flux_smooth(st[m2], a.gas, STAGE == 1, F, dF);
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            if (STAGE == 1) Fs[i] += F[i];
            Fs[5 + i] += dF[i];
          }
        }
      }
    } else if constexpr (FLUX == FLUX_FULL && TPF == 2) {
      // Full flux, two threads per face: thread `sub` takes the t1 abscissa
      // m1 = sub; one pass along t2 per field gives both t2 abscissae.  The
      // point states of m2 = 1 wait in the thread's shared-memory slots
      // (index ((s*4 + c)*5 + i)*256 + tid, c = 0 value, 1..3 derivatives
      // along n, t1, t2) while the flux at m2 = 0 is evaluated.
      static_assert(NT == 256, "the shared-memory slots are laid out for 256 threads");
      const int m1 = sub;
      PointState<T> st[3];
      // One state group per iteration (the loop body once in the code): the
      // group's m2 = 0 states go to st[s] through constant indices.
#pragma unroll 1
      for (int s = 0; s < 3; ++s) {
        PointState<T> g0;
        if constexpr (is_char_mode<MODE>()) {
          T val[2][5], d2[2][5], d1[2][5], dn[2][5];
          t2_group<T, MODE, NV, NH>(tb, s, m1, at3, st2, cbs, val, d2, d1, dn);
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            g0.q[i] = val[0][i];
            g0.dq[0][i] = dn[0][i];
            g0.dq[1][i] = d1[0][i] * rh1;
            g0.dq[2][i] = d2[0][i] * rh2;
            scr[((s * 4 + 0) * 5 + i) * 256 + tid] = val[1][i];
            scr[((s * 4 + 1) * 5 + i) * 256 + tid] = dn[1][i];
            scr[((s * 4 + 2) * 5 + i) * 256 + tid] = d1[1][i] * rh1;
            scr[((s * 4 + 3) * 5 + i) * 256 + tid] = d2[1][i] * rh2;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            const int k = 5 * s + i;
            const T* sv = tb + (4 * k + m1) * NH + at3;
            const T* sdv = tb + (4 * k + 2 + m1) * NH + at3;
            const T* ss = tb + (4 * NV + 2 * k + m1) * NH + at3;
            T v[2], dd[2], vd[2], vs[2];
            tangential<MODE>(sv[-2 * st2], sv[-st2], sv[0], sv[st2], sv[2 * st2], v, dd);
            tangential_val<MODE>(sdv[-2 * st2], sdv[-st2], sdv[0], sdv[st2], sdv[2 * st2], vd);
            tangential_val<MODE>(ss[-2 * st2], ss[-st2], ss[0], ss[st2], ss[2 * st2], vs);
            g0.q[i] = v[0];
            g0.dq[0][i] = vs[0];
            g0.dq[1][i] = vd[0] * rh1;
            g0.dq[2][i] = dd[0] * rh2;
            scr[((s * 4 + 0) * 5 + i) * 256 + tid] = v[1];
            scr[((s * 4 + 1) * 5 + i) * 256 + tid] = vs[1];
            scr[((s * 4 + 2) * 5 + i) * 256 + tid] = vd[1] * rh1;
            scr[((s * 4 + 3) * 5 + i) * 256 + tid] = dd[1] * rh2;
          }
        }
        if (s == 0) st[0] = g0;
        else if (s == 1) st[1] = g0;
        else st[2] = g0;
      }
#pragma unroll 1
      for (int m2 = 0; m2 < 2; ++m2) {
        if (m2 == 1) {
#pragma unroll
          for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              st[s].q[i] = scr[((s * 4 + 0) * 5 + i) * 256 + tid];
              st[s].dq[0][i] = scr[((s * 4 + 1) * 5 + i) * 256 + tid];
              st[s].dq[1][i] = scr[((s * 4 + 2) * 5 + i) * 256 + tid];
              st[s].dq[2][i] = scr[((s * 4 + 3) * 5 + i) * 256 + tid];
            }
        }
        T F[5], dF[5];
        flux_full(st[0], st[1], st[2], a.gas, dt, F, dF);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          if (STAGE == 1) Fs[i] += F[i];
          Fs[5 + i] += dF[i];
        }
      }
    } else {
#pragma unroll 1
      for (int g = sub * GPF; g < (sub + 1) * GPF; ++g) {
        const int m1 = g & 1, m2 = g >> 1;
        constexpr int NS = FLUX == FLUX_FULL ? 3 : 1;
        PointState<T> st[NS];
        // One state group per iteration (the body once in the code); the
        // group's states go to st[s] through constant indices.
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
          PointState<T> g0;
          if constexpr (is_char_mode<MODE>()) {
            T val[2][5], d2[2][5], d1[2][5], dn[2][5];
            t2_group<T, MODE, NV, NH>(tb, s, m1, at3, st2, cbs, val, d2, d1, dn);
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              g0.q[i] = val[m2][i];
              g0.dq[0][i] = dn[m2][i];
              g0.dq[1][i] = d1[m2][i] * rh1;
              g0.dq[2][i] = d2[m2][i] * rh2;
            }
          } else {
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              const int k = 5 * s + i;
              const T* sv = tb + (4 * k + m1) * NH + at3;
              const T* sdv = tb + (4 * k + 2 + m1) * NH + at3;
              const T* ss = tb + (4 * NV + 2 * k + m1) * NH + at3;
              T v[2], dd[2];
              tangential<MODE>(sv[-2 * st2], sv[-st2], sv[0], sv[st2], sv[2 * st2], v, dd);
              g0.q[i] = v[m2];
              g0.dq[2][i] = dd[m2] * rh2;
              tangential_val<MODE>(sdv[-2 * st2], sdv[-st2], sdv[0], sdv[st2], sdv[2 * st2], v);
              g0.dq[1][i] = v[m2] * rh1;
              tangential_val<MODE>(ss[-2 * st2], ss[-st2], ss[0], ss[st2], ss[2 * st2], v);
              g0.dq[0][i] = v[m2];
            }
          }
          if (s == 0) st[0] = g0;
          else if (NS > 1 && s == 1) st[NS > 1 ? 1 : 0] = g0;
          else if (NS > 2) st[NS > 2 ? 2 : 0] = g0;
        }
        T F[5], dF[5];
        if constexpr (FLUX == FLUX_SMOOTH) {
          flux_smooth(st[0], a.gas, STAGE == 1, F, dF);
        } else {
          flux_full(st[0], st[1], st[2], a.gas, dt, F, dF);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          if (STAGE == 1) Fs[i] += F[i];
          Fs[5 + i] += dF[i];
        }
      }
    }
    if (TPF > 1 && sub > 0) {
#pragma unroll
      for (int i = 0; i < 10; ++i) part[((sub - 1) * 10 + i) * NFACE + face] = Fs[i];
    }
    if (TPF > 1) __syncthreads();
    if (sub == 0 && f_valid) {
#pragma unroll
      for (int r = 1; r < TPF; ++r)
#pragma unroll
        for (int i = 0; i < 10; ++i) Fs[i] += part[((r - 1) * 10 + i) * NFACE + face];
      const long long o = fout + (long long)f * fstep;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        // The second stage needs dF only (Eq. (6)); its F planes are not written.
        if (STAGE == 1) a.fd[ax.gv[i] * FS + o] = T(0.25) * Fs[i];
        a.fd[(5 + ax.gv[i]) * FS + o] = T(0.25) * Fs[5 + i];
      }
    }
    __syncthreads();
  }
  }
}

}  // namespace hgks

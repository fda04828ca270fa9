// HGKS oracle: a plain, slow FP64 CPU restatement of one time step of the
// high-order gas-kinetic scheme (HGKS) of Cao, Pan & Xu, "High-order
// gas-kinetic scheme with parallel computation for direct numerical
// simulation of turbulent flows" (arXiv:2005.08736).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py load this library.  It shares no
// code, header, table or constant generator with the CUDA path in
// paper_2005_08736_gb300/, and it never calls that path.
//
// The code follows the paper's steps in the paper's order and notation:
//   Sec. 2.1, Eq. (1)-(2)  BGK model, Maxwellian g, compatibility condition
//   Sec. 2.1, Eq. (3)-(4)  finite-volume semi-discretisation, 2x2 Gauss points
//   Sec. 2.1, Eq. (5)      second-order distribution f at a Gauss point, the
//                          compatibility Q0 and the slope / time conditions
//   Sec. 2.1, Remark 1     WENO5 (linear weights / WENO-JS / WENO-Z) normal
//                          reconstruction and the tangential reconstruction
//   Sec. 2.1, Eq. (6)-(7)  two-stage fourth-order (S2O4) update and the linear
//                          flux fit over [0, dt/2] and [0, dt]
//   Sec. 3 (opening)       collision time tau = mu/p (+ numerical term)
//   Sec. 3.3               tanh channel mapping, isothermal no-slip walls,
//                          streamwise body force
// Points the paper leaves open are marked "Reading:"; the same readings are
// followed by the CUDA path.  Moments are evaluated generically: every needed
// velocity-space integral is written as a product of polynomials in
// (u, v, w, xi^2) and integrated monomial by monomial against the
// Maxwellian, which factorises over u, v, w and xi.  Linear solves use plain
// Gaussian elimination.  Nothing is fused or reordered for speed.
//
// Units: gas constant R = 1, so p = rho T and lambda = rho / (2 p).
// Layout of every field array crossing the C interface: [5][nz][ny][nx],
// x fastest, variables (rho, rho U, rho V, rho W, rho E).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// Scalar type of every quantity that depends on the state.  The plain build
// computes in double.  The tangent build (-DORACLE_TANGENT) computes in the
// forward-mode dual numbers of tangent.h: the same code then also carries the
// derivative along one input direction (a dual-number tangent run), while its
// value part repeats the double arithmetic of the plain build exactly.  The
// counting build (-DORACLE_COUNT) computes in the tallying doubles of
// counted.h: the same values, plus the number of operations performed.
// Configuration constants, cell widths, the Gauss abscissae and dt stay double
// (dt is held fixed when differentiating, as in the adjoint).
#if defined(ORACLE_TANGENT)
#include "tangent.h"
using real = oracle_dual::Dual;
using oracle_dual::value;
#elif defined(ORACLE_COUNT)
#include "counted.h"
using real = oracle_count::Counted;
using oracle_count::value;
#else
using real = double;
inline double value(double x) { return x; }
#endif
using std::erfc;
using std::exp;
using std::fabs;
using std::pow;
using std::sqrt;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int G = 3;  // ghost layers on every side

// ---------------------------------------------------------------------------
// Polynomials in the particle velocity (u, v, w) and xi^2.
// ---------------------------------------------------------------------------
struct Mono {
  real c;
  int a, b, w, d;  // c * u^a v^b w^w (xi^2)^d
};
struct Poly {
  int n = 0;
  Mono m[24];
  void add(real c, int a, int b, int w, int d) { m[n++] = Mono{c, a, b, w, d}; }
};

// psi = (1, u, v, w, (u^2 + v^2 + w^2 + xi^2)/2), Sec. 2.1 after Eq. (2).
Poly psi(int i) {
  Poly p;
  switch (i) {
    case 0: p.add(1, 0, 0, 0, 0); break;
    case 1: p.add(1, 1, 0, 0, 0); break;
    case 2: p.add(1, 0, 1, 0, 0); break;
    case 3: p.add(1, 0, 0, 1, 0); break;
    default:
      p.add(0.5, 2, 0, 0, 0);
      p.add(0.5, 0, 2, 0, 0);
      p.add(0.5, 0, 0, 2, 0);
      p.add(0.5, 0, 0, 0, 1);
  }
  return p;
}

// Velocity component u_d (d = 0: u, 1: v, 2: w) as a polynomial.
Poly vel(int d) {
  Poly p;
  p.add(1, d == 0, d == 1, d == 2, 0);
  return p;
}

// a . psi = a1 + a2 u + a3 v + a4 w + a5 (u^2+v^2+w^2+xi^2)/2.
Poly lin(const real a[5]) {
  Poly p;
  p.add(a[0], 0, 0, 0, 0);
  p.add(a[1], 1, 0, 0, 0);
  p.add(a[2], 0, 1, 0, 0);
  p.add(a[3], 0, 0, 1, 0);
  p.add(0.5 * a[4], 2, 0, 0, 0);
  p.add(0.5 * a[4], 0, 2, 0, 0);
  p.add(0.5 * a[4], 0, 0, 2, 0);
  p.add(0.5 * a[4], 0, 0, 0, 1);
  return p;
}

// Peculiar heat-flux density h = c_u (c_u^2 + c_v^2 + c_w^2 + xi^2) / 2 with
// c = (u - U, v - V, w - W), expanded into monomials.
Poly heat(real U, real V, real W) {
  Poly p;
  // (u-U)^3 / 2
  p.add(0.5, 3, 0, 0, 0);
  p.add(-1.5 * U, 2, 0, 0, 0);
  p.add(1.5 * U * U, 1, 0, 0, 0);
  p.add(-0.5 * U * U * U, 0, 0, 0, 0);
  // (u-U)(v-V)^2 / 2 and (u-U)(w-W)^2 / 2
  const real T[2] = {V, W};
  for (int s = 0; s < 2; ++s) {
    const real C = T[s];
    const int b2 = s == 0 ? 2 : 0, w2 = s == 0 ? 0 : 2;
    const int b1 = s == 0 ? 1 : 0, w1 = s == 0 ? 0 : 1;
    p.add(0.5, 1, b2, w2, 0);
    p.add(-C, 1, b1, w1, 0);
    p.add(0.5 * C * C, 1, 0, 0, 0);
    p.add(-0.5 * U, 0, b2, w2, 0);
    p.add(U * C, 0, b1, w1, 0);
    p.add(-0.5 * U * C * C, 0, 0, 0, 0);
  }
  // (u-U) xi^2 / 2
  p.add(0.5, 1, 0, 0, 1);
  p.add(-0.5 * U, 0, 0, 0, 1);
  return p;
}

// ---------------------------------------------------------------------------
// Maxwellian g = rho (lambda/pi)^((K+3)/2) exp(-lambda((u-U)^2+(v-V)^2+(w-W)^2+xi^2))
// (Sec. 2.1, Eq. (1)) and its normalised moments <.> = (1/rho) int g (.) dXi.
// ---------------------------------------------------------------------------
constexpr int kMaxDeg = 10;

struct Maxwellian {
  real rho, U, V, W, lam;
  real uf[kMaxDeg], up[kMaxDeg], un[kMaxDeg];  // <u^n>: full, u>0, u<0
  real v[kMaxDeg], w[kMaxDeg];                  // <v^n>, <w^n>
  real xi[4];                                   // <(xi^2)^m>
};

// One-dimensional Gaussian moments by the recursion
//   <u^(n+2)> = U <u^(n+1)> + (n+1)/(2 lambda) <u^n>,
// which holds over the whole line and over each half line (integration by
// parts; the boundary term at u = 0 vanishes for n >= 0).
void recur(real* m, real U, real lam) {
  for (int n = 0; n + 2 < kMaxDeg; ++n)
    m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

void set_moments(Maxwellian& g, double K) {
  const real lam = g.lam;
  g.uf[0] = 1.0;
  g.uf[1] = g.U;
  recur(g.uf, g.U, lam);
  g.v[0] = 1.0;
  g.v[1] = g.V;
  recur(g.v, g.V, lam);
  g.w[0] = 1.0;
  g.w[1] = g.W;
  recur(g.w, g.W, lam);
  // Half-space moments: <u^0>_{u>0} = erfc(-sqrt(lambda) U)/2,
  // <u^1>_{u>0} = U <u^0>_{u>0} + exp(-lambda U^2) / (2 sqrt(pi lambda)).
  const real s = sqrt(lam);
  const real e = exp(-lam * g.U * g.U) / (2.0 * sqrt(kPi * lam));
  g.up[0] = 0.5 * erfc(-s * g.U);
  g.up[1] = g.U * g.up[0] + e;
  recur(g.up, g.U, lam);
  g.un[0] = 0.5 * erfc(s * g.U);
  g.un[1] = g.U * g.un[0] - e;
  recur(g.un, g.U, lam);
  // Internal degrees of freedom: xi^2 = sum of K squares, each of variance
  // 1/(2 lambda), so <(xi^2)^m> = K (K+2) ... (K+2m-2) / (2 lambda)^m.
  g.xi[0] = 1.0;
  for (int m = 1; m < 4; ++m) g.xi[m] = g.xi[m - 1] * (K + 2.0 * (m - 1)) / (2.0 * lam);
}

// Primitive state and moments from a conservative state in the local frame.
Maxwellian maxwellian(const real Q[5], double gamma) {
  Maxwellian g;
  const double K = (5.0 - 3.0 * gamma) / (gamma - 1.0);  // Sec. 2.1: N = (5-3 gamma)/(gamma-1)
  g.rho = Q[0];
  g.U = Q[1] / Q[0];
  g.V = Q[2] / Q[0];
  g.W = Q[3] / Q[0];
  const real p = (gamma - 1.0) * (Q[4] - 0.5 * Q[0] * (g.U * g.U + g.V * g.V + g.W * g.W));
  g.lam = Q[0] / (2.0 * p);
  set_moments(g, K);
  return g;
}

// <product of the given polynomials>, half = 0 whole space, +1 u > 0, -1 u < 0.
real mom(const Maxwellian& g, int half, const Poly* const* f, int nf) {
  const real* um = half == 0 ? g.uf : (half > 0 ? g.up : g.un);
  real sum = 0.0;
  int idx[4] = {0, 0, 0, 0};
  while (true) {
    real c = 1.0;
    int a = 0, b = 0, w = 0, d = 0;
    for (int k = 0; k < nf; ++k) {
      const Mono& m = f[k]->m[idx[k]];
      c *= m.c;
      a += m.a;
      b += m.b;
      w += m.w;
      d += m.d;
    }
    if (c != 0.0) sum += c * um[a] * g.v[b] * g.w[w] * g.xi[d];
    int k = nf - 1;
    while (k >= 0 && ++idx[k] == f[k]->n) idx[k--] = 0;
    if (k < 0) break;
  }
  return sum;
}
real mom(const Maxwellian& g, int half, const Poly& A) {
  const Poly* f[1] = {&A};
  return mom(g, half, f, 1);
}
real mom(const Maxwellian& g, int half, const Poly& A, const Poly& B) {
  const Poly* f[2] = {&A, &B};
  return mom(g, half, f, 2);
}
real mom(const Maxwellian& g, int half, const Poly& A, const Poly& B, const Poly& C) {
  const Poly* f[3] = {&A, &B, &C};
  return mom(g, half, f, 3);
}
real mom(const Maxwellian& g, int half, const Poly& A, const Poly& B, const Poly& C,
           const Poly& D) {
  const Poly* f[4] = {&A, &B, &C, &D};
  return mom(g, half, f, 4);
}

// Dense Gaussian elimination with partial pivoting, n <= 8.
template <class S>
void gauss_solve(int n, S* A, S* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const S f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    S s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
}

// Slope coefficients: the a in <a . psi> = dQ / rho, i.e. the solution of
// M a = b with M_ij = <psi_i psi_j>  (Sec. 2.1, conditions below Eq. (5)).
void slope_solve(const Maxwellian& g, const real b[5], real a[5]) {
  real M[25], r[5];
  for (int i = 0; i < 5; ++i) {
    const Poly pi = psi(i);
    for (int j = 0; j < 5; ++j) M[i * 5 + j] = mom(g, 0, pi, psi(j));
    r[i] = b[i];
  }
  gauss_solve(5, M, r);
  for (int i = 0; i < 5; ++i) a[i] = r[i];
}

// Derived kinetic data of one reconstructed state at a Gauss point.
struct Kin {
  Maxwellian g;
  real a[3][5];  // spatial slopes along n, t1, t2 (local frame)
  real A[5];     // time coefficient
};

// Slopes from <a_d> = dQ/dx_d and A from <a_1 u + a_2 v + a_3 w + A> = 0,
// all moments of the state's own Maxwellian (Sec. 2.1, below Eq. (5)).
Kin kinetic(const real Q[5], const real dQ[3][5], double gamma) {
  Kin k;
  k.g = maxwellian(Q, gamma);
  for (int d = 0; d < 3; ++d) {
    real b[5];
    for (int i = 0; i < 5; ++i) b[i] = dQ[d][i] / Q[0];
    slope_solve(k.g, b, k.a[d]);
  }
  real rhs[5];
  for (int i = 0; i < 5; ++i) {
    const Poly pi = psi(i);
    real s = 0.0;
    for (int d = 0; d < 3; ++d) s += mom(k.g, 0, lin(k.a[d]), vel(d), pi);
    rhs[i] = -s;
  }
  slope_solve(k.g, rhs, k.A);
  return k;
}

// <u psi_i>, <u (a_n.psi u + a_t1.psi v + a_t2.psi w) psi_i>, <u (A.psi) psi_i>.
real m_u(const Maxwellian& g, int half, int i) { return mom(g, half, vel(0), psi(i)); }
real m_ua(const Maxwellian& g, int half, const real a[3][5], int i) {
  real s = 0.0;
  for (int d = 0; d < 3; ++d) s += mom(g, half, vel(0), lin(a[d]), vel(d), psi(i));
  return s;
}
real m_uA(const Maxwellian& g, int half, const real A[5], int i) {
  return mom(g, half, vel(0), lin(A), psi(i));
}

// Time integrals over [0, T] of the five coefficients of Eq. (5), e = exp(-T/tau).
void time_integrals(double T, real tau, real q[6]) {
  const real e = exp(-T / tau);
  q[0] = T - tau * (1.0 - e);                                   // (1 - e^{-t/tau})
  q[1] = 2.0 * tau * tau * (1.0 - e) - tau * T * (1.0 + e);    // (t+tau) e^{-t/tau} - tau
  q[2] = 0.5 * T * T - tau * T + tau * tau * (1.0 - e);        // t - tau + tau e^{-t/tau}
  q[3] = tau * (1.0 - e);                                       // e^{-t/tau}
  q[4] = tau * (T * e - 2.0 * tau * (1.0 - e));                // -(tau + t) e^{-t/tau}
  q[5] = -tau * tau * (1.0 - e);                                // -tau e^{-t/tau}
}

// ---------------------------------------------------------------------------
// Reconstruction (Sec. 2.1, Remark 1).
// ---------------------------------------------------------------------------
enum { RECON_LINEAR = 0, RECON_WENO_JS = 1, RECON_WENO_Z = 2 };
enum { FLUX_SMOOTH = 0, FLUX_FULL = 1 };

// Fifth-order WENO value at the right end of the centre cell of q[0..4]
// (cell averages q_{i-2} .. q_{i+2}): the three third-order candidates on the
// stencils {i-2,i-1,i}, {i-1,i,i+1}, {i,i+1,i+2}, the optimal linear weights
// (1/10, 6/10, 3/10), and the Jiang-Shu smoothness indicators.
// Reading: WENO-JS uses eps = 1e-6 and power 2; WENO-Z uses
// tau5 = |beta0 - beta2|, alpha_k = d_k (1 + tau5 / (beta_k + eps)), eps = 1e-20.
real weno5_right(const real q[5], int mode) {
  const real p0 = (2.0 * q[0] - 7.0 * q[1] + 11.0 * q[2]) / 6.0;
  const real p1 = (-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.0;
  const real p2 = (2.0 * q[2] + 5.0 * q[3] - q[4]) / 6.0;
  const real d[3] = {0.1, 0.6, 0.3};
  real w[3] = {d[0], d[1], d[2]};
  if (mode != RECON_LINEAR) {
    const real s0 = q[0] - 2.0 * q[1] + q[2], t0 = q[0] - 4.0 * q[1] + 3.0 * q[2];
    const real s1 = q[1] - 2.0 * q[2] + q[3], t1 = q[1] - q[3];
    const real s2 = q[2] - 2.0 * q[3] + q[4], t2 = 3.0 * q[2] - 4.0 * q[3] + q[4];
    const real beta[3] = {13.0 / 12.0 * s0 * s0 + 0.25 * t0 * t0,
                            13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1,
                            13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2};
    real alpha[3], sum = 0.0;
    for (int k = 0; k < 3; ++k) {
      if (mode == RECON_WENO_JS) {
        alpha[k] = d[k] / ((1e-6 + beta[k]) * (1e-6 + beta[k]));
      } else {
        const real tau5 = fabs(beta[0] - beta[2]);
        alpha[k] = d[k] * (1.0 + tau5 / (beta[k] + 1e-20));
      }
      sum += alpha[k];
    }
    for (int k = 0; k < 3; ++k) w[k] = alpha[k] / sum;
  }
  return w[0] * p0 + w[1] * p1 + w[2] * p2;
}
// Value at the left end of the centre cell: the mirrored stencil.
real weno5_left(const real q[5], int mode) {
  const real r[5] = {q[4], q[3], q[2], q[1], q[0]};
  return weno5_right(r, mode);
}

// Gauss abscissae of the two-point rule in cell units, s in [-1/2, 1/2].
const double kGaussS[2] = {-0.5 / std::sqrt(3.0), 0.5 / std::sqrt(3.0)};

// Weights of the quartic tangential reconstruction (Remark 1, smooth flows):
// the fourth-degree polynomial P(s) whose averages over the five cells
// [k-1/2, k+1/2], k = -2..2, equal the data; wv[m][k] gives P(s_m), wd[m][k]
// gives P'(s_m) (cell units).  Built once by solving the 5x5 system of
// monomial averages.
struct QuarticWeights {
  double wv[2][5], wd[2][5];
  QuarticWeights() {
    for (int k = 0; k < 5; ++k) {
      // Solve for the polynomial reproducing the unit vector e_k.
      double A[25], c[5];
      for (int r = 0; r < 5; ++r) {
        const double lo = (r - 2) - 0.5, hi = (r - 2) + 0.5;
        for (int p = 0; p < 5; ++p) A[r * 5 + p] = (std::pow(hi, p + 1) - std::pow(lo, p + 1)) / (p + 1);
        c[r] = (r == k) ? 1.0 : 0.0;
      }
      gauss_solve(5, A, c);
      for (int m = 0; m < 2; ++m) {
        const double s = kGaussS[m];
        double v = 0.0, dv = 0.0;
        for (int p = 0; p < 5; ++p) {
          v += c[p] * std::pow(s, p);
          if (p > 0) dv += p * c[p] * std::pow(s, p - 1);
        }
        wv[m][k] = v;
        wd[m][k] = dv;
      }
    }
  }
};
const QuarticWeights& quartic() {
  static const QuarticWeights w;
  return w;
}

// Tangential reconstruction of a face field from five face averages f[0..4]
// (cells j-2..j+2 of the tangential direction): values val[m] and
// derivatives der[m] (per unit cell length) at the two Gauss abscissae of cell j.
// LINEAR: the quartic above.  WENO modes (Remark 1, last paragraph): WENO5
// values at both ends of cell j plus its average define the quadratic
// p(s) = a + b s + c s^2 with b = QR - QL, c = 3(QL + QR) - 6 f_j, a = f_j - c/12.
void tangential(const real f[5], int mode, real val[2], real der[2]) {
  if (mode == RECON_LINEAR) {
    const QuarticWeights& W = quartic();
    for (int m = 0; m < 2; ++m) {
      val[m] = der[m] = 0.0;
      for (int k = 0; k < 5; ++k) {
        val[m] += W.wv[m][k] * f[k];
        der[m] += W.wd[m][k] * f[k];
      }
    }
    return;
  }
  const real QL = weno5_left(f, mode), QR = weno5_right(f, mode);
  const real b = QR - QL, c = 3.0 * (QL + QR) - 6.0 * f[2], a = f[2] - c / 12.0;
  for (int m = 0; m < 2; ++m) {
    const real s = kGaussS[m];
    val[m] = a + b * s + c * s * s;
    der[m] = b + 2.0 * c * s;
  }
}

// ---------------------------------------------------------------------------
// Characteristic variables (Sec. 2.1, Remark 1): omega = R^{-1} Q, with R the
// right eigenvectors of the Jacobian dF/dQ of the Euler flux along the local
// normal (velocity component 1 of the local frame), taken at a state Qm.
// Columns of R, for the eigenvalues u - c, u, u, u, u + c:
//   (1, u - c, v, w, H - u c), (1, u, v, w, |U|^2 / 2), (0, 0, 1, 0, v),
//   (0, 0, 0, 1, w), (1, u + c, v, w, H + u c);
// H = (rho E + p)/rho, c^2 = gamma p / rho.  R^{-1} is formed by Gaussian
// elimination.
// ---------------------------------------------------------------------------
struct CharBasis {
  real R[5][5];
  real L[5][5];
};

CharBasis char_basis(const real Qm[5], double gamma) {
  const real rho = Qm[0], u = Qm[1] / rho, v = Qm[2] / rho, w = Qm[3] / rho;
  const real q2 = u * u + v * v + w * w;
  const real p = (gamma - 1.0) * (Qm[4] - 0.5 * rho * q2);
  const real c = sqrt(gamma * p / rho), H = (Qm[4] + p) / rho;
  const real cols[5][5] = {{1.0, u - c, v, w, H - u * c},
                             {1.0, u, v, w, 0.5 * q2},
                             {0.0, 0.0, 1.0, 0.0, v},
                             {0.0, 0.0, 0.0, 1.0, w},
                             {1.0, u + c, v, w, H + u * c}};
  CharBasis B;
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) B.R[i][k] = cols[k][i];
  for (int k = 0; k < 5; ++k) {  // column k of R^{-1}: R x = e_k
    real A[25], e[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) A[i * 5 + j] = B.R[i][j];
    e[k] = 1.0;
    gauss_solve(5, A, e);
    for (int i = 0; i < 5; ++i) B.L[i][k] = e[i];
  }
  return B;
}

void mat5(const real M[5][5], const real x[5], real y[5]) {
  for (int i = 0; i < 5; ++i) {
    y[i] = 0.0;
    for (int k = 0; k < 5; ++k) y[i] += M[i][k] * x[k];
  }
}

// Tangential reconstruction of a 5-vector field from the five face averages
// f[s][0..4] (Remark 1), component-wise or, with B, in the characteristic
// variables of B: project every average, reconstruct each characteristic
// component, map the values and derivatives back.
void tangential_vec(const real f[5][5], int mode, const CharBasis* B, real val[2][5],
                    real der[2][5]) {
  real g[5][5];
  for (int s = 0; s < 5; ++s) {
    if (B) mat5(B->L, f[s], g[s]);
    else
      for (int i = 0; i < 5; ++i) g[s][i] = f[s][i];
  }
  real cv[2][5], cd[2][5];
  for (int i = 0; i < 5; ++i) {
    const real col[5] = {g[0][i], g[1][i], g[2][i], g[3][i], g[4][i]};
    real v2[2], d2[2];
    tangential(col, mode, v2, d2);
    for (int m = 0; m < 2; ++m) {
      cv[m][i] = v2[m];
      cd[m][i] = d2[m];
    }
  }
  for (int m = 0; m < 2; ++m) {
    if (B) {
      mat5(B->R, cv[m], val[m]);
      mat5(B->R, cd[m], der[m]);
    } else {
      for (int i = 0; i < 5; ++i) {
        val[m][i] = cv[m][i];
        der[m][i] = cd[m][i];
      }
    }
  }
}

// Normal WENO5 end values of cells i = f-1 (stencil qc[0..4]) and i+1 = f
// (qc[1..5]): out[0] = Q at x_{i+1/2} from cell i, out[1] = Q at x_{i-1/2}
// from cell i, out[2] = Q at x_{i+1/2} from cell i+1, out[3] = Q at x_{i+3/2}
// from cell i+1; component-wise or in the characteristic variables of B.
void normal_end_values(const real qc[6][5], int mode, const CharBasis* B, real out[4][5]) {
  real g[6][5];
  for (int s = 0; s < 6; ++s) {
    if (B) mat5(B->L, qc[s], g[s]);
    else
      for (int i = 0; i < 5; ++i) g[s][i] = qc[s][i];
  }
  real e[4][5];
  for (int i = 0; i < 5; ++i) {
    const real sl[5] = {g[0][i], g[1][i], g[2][i], g[3][i], g[4][i]};
    const real sr[5] = {g[1][i], g[2][i], g[3][i], g[4][i], g[5][i]};
    e[0][i] = weno5_right(sl, mode);
    e[1][i] = weno5_left(sl, mode);
    e[2][i] = weno5_left(sr, mode);
    e[3][i] = weno5_right(sr, mode);
  }
  for (int k = 0; k < 4; ++k) {
    if (B) mat5(B->R, e[k], out[k]);
    else
      for (int i = 0; i < 5; ++i) out[k][i] = e[k][i];
  }
}

// ---------------------------------------------------------------------------
// Configuration and the flux at one Gauss point.
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {

// Oracle configuration (its own definition; the CUDA library has another).
typedef struct {
  int nx, ny, nz;
  double x0, lx, y0, ly, z0, lz;
  int y_stretch;     // 0 uniform, 1 tanh mapping of Sec. 3.3
  double stretch_b;  // b_g of the mapping
  int bc_y;          // 0 periodic, 1 isothermal no-slip walls at both y ends
  double gamma, prandtl;
  int visc_law;      // 0 constant mu = mu_ref, 1 mu = mu_ref (T/T_ref)^visc_exp
  double mu_ref, T_ref, visc_exp;
  double T_wall, force_x;
  int recon, flux;   // RECON_*, FLUX_*
  double tau_num_C;  // C of the numerical collision time (Sec. 3); 0 disables
  double cfl;
  int force_mode;    // 0 the constant force_x; 1 the constant-mass-flux force of Sec. 3.3
  double mass_flux;  // force_mode 1: the volume average of rho U that the force keeps
  int char_recon;    // 1: reconstruct characteristic variables (Remark 1); 0: conservative
} oracle_config;

}  // extern "C"

namespace {

real viscosity(const oracle_config& c, real T) {
  if (c.visc_law == 0) return c.mu_ref;
  return c.mu_ref * pow(T / c.T_ref, c.visc_exp);
}

// Reconstructed data at one Gauss point, local frame (normal velocity first):
// st[s][0] value, st[s][1..3] derivatives along n, t1, t2, for s = l, r, 0.
struct PointData {
  real st[3][4][5];
};

// Numerical flux density at one Gauss point: F (time-averaged flux of the
// linear fit, Eq. (7)) and dF (its time derivative), local frame.
void flux_point(const oracle_config& c, const PointData& pd, double dt, real F[5],
                real dF[5]) {
  real dQ[3][5];
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 5; ++i) dQ[d][i] = pd.st[2][d + 1][i];
  const Kin k0 = kinetic(pd.st[2][0], dQ, c.gamma);
  const Maxwellian& g0 = k0.g;
  // Collision time (Sec. 3): tau = mu/p with p the interface (g0) pressure;
  // the full flux adds C |p_l - p_r| / (p_l + p_r) dt.
  const real p0 = g0.rho / (2.0 * g0.lam);
  real tau = viscosity(c, 1.0 / (2.0 * g0.lam)) / p0;

  if (c.flux == FLUX_SMOOTH) {
    // Simplified smooth flux (Remark 1): f = g0 [1 - tau (abar.u + Abar) + t Abar].
    for (int i = 0; i < 5; ++i) {
      F[i] = g0.rho * (m_u(g0, 0, i) - tau * (m_ua(g0, 0, k0.a, i) + m_uA(g0, 0, k0.A, i)));
      dF[i] = g0.rho * m_uA(g0, 0, k0.A, i);
    }
  } else {
    real dQl[3][5], dQr[3][5];
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < 5; ++i) {
        dQl[d][i] = pd.st[0][d + 1][i];
        dQr[d][i] = pd.st[1][d + 1][i];
      }
    const Kin kl = kinetic(pd.st[0][0], dQl, c.gamma);
    const Kin kr = kinetic(pd.st[1][0], dQr, c.gamma);
    const real pl = kl.g.rho / (2.0 * kl.g.lam), pr = kr.g.rho / (2.0 * kr.g.lam);
    tau += c.tau_num_C * fabs((pl - pr) / (pl + pr)) * dt;
    // Time-integrated flux W(T) of Eq. (5).  Reading: the Heaviside factor
    // H(u) (u > 0) belongs to g_l and 1 - H(u) to g_r, as in the compatibility
    // condition for Q0 printed below Eq. (5).
    // Moment vectors of the three parts of f, then W(T) for T = dt, dt/2.
    real m0[3][5], ml[3][5], mr[3][5];
    for (int i = 0; i < 5; ++i) {
      m0[0][i] = g0.rho * m_u(g0, 0, i);
      m0[1][i] = g0.rho * m_ua(g0, 0, k0.a, i);
      m0[2][i] = g0.rho * m_uA(g0, 0, k0.A, i);
      ml[0][i] = kl.g.rho * m_u(kl.g, +1, i);
      ml[1][i] = kl.g.rho * m_ua(kl.g, +1, kl.a, i);
      ml[2][i] = kl.g.rho * m_uA(kl.g, +1, kl.A, i);
      mr[0][i] = kr.g.rho * m_u(kr.g, -1, i);
      mr[1][i] = kr.g.rho * m_ua(kr.g, -1, kr.a, i);
      mr[2][i] = kr.g.rho * m_uA(kr.g, -1, kr.A, i);
    }
    real W[2][5];
    const double Ts[2] = {dt, 0.5 * dt};
    for (int t = 0; t < 2; ++t) {
      real q[6];
      time_integrals(Ts[t], tau, q);
      for (int i = 0; i < 5; ++i)
        W[t][i] = q[0] * m0[0][i] + q[1] * m0[1][i] + q[2] * m0[2][i] +
                  q[3] * (ml[0][i] + mr[0][i]) + q[4] * (ml[1][i] + mr[1][i]) +
                  q[5] * (ml[2][i] + mr[2][i]);
    }
    // Linear fit F(t) = F + dF t (Eq. (7)) from W(dt) and W(dt/2).
    for (int i = 0; i < 5; ++i) {
      F[i] = (4.0 * W[1][i] - W[0][i]) / dt;
      dF[i] = 4.0 * (W[0][i] - 2.0 * W[1][i]) / (dt * dt);
    }
  }
  // Reading (Prandtl number, Sec. 3.1 gives Pr but not the mechanism): the
  // BGK model has Pr = 1; the energy flux F gets (1/Pr - 1) times the heat
  // flux of the non-equilibrium part -tau (abar.u + Abar) g0, measured in the
  // frame of g0.  dF is left unchanged.
  if (c.prandtl != 1.0) {
    const Poly h = heat(g0.U, g0.V, g0.W);
    real q = 0.0;
    for (int d = 0; d < 3; ++d) q += mom(g0, 0, h, lin(k0.a[d]), vel(d));
    q += mom(g0, 0, h, lin(k0.A));
    q *= -tau * g0.rho;
    F[4] += (1.0 / c.prandtl - 1.0) * q;
  }
}

// Two-stage fourth-order update, Eq. (6):
//   Q*      = Q^n + dt/2 L(Q^n) + dt^2/8 dL(Q^n)
//   Q^{n+1} = Q^n + dt L(Q^n) + dt^2/6 (dL(Q^n) + 2 dL(Q*)).
real s2o4_stage1(real Qn, real L0, real dL0, double dt) {
  return Qn + 0.5 * dt * L0 + 0.125 * dt * dt * dL0;
}
real s2o4_stage2(real Qn, real L0, real dL0, real dL1, double dt) {
  return Qn + dt * L0 + dt * dt / 6.0 * (dL0 + 2.0 * dL1);
}

// ---------------------------------------------------------------------------
// The solver: padded state with G ghost layers, one S2O4 step.
// ---------------------------------------------------------------------------
struct Solver {
  oracle_config c;
  int n[3];
  int pn[3];                       // padded sizes
  std::vector<double> width[3];    // cell widths, index -G .. n+G-1 (offset G)
  std::vector<real> q;           // padded conservative state [5][pz][py][px]
  double t = 0.0;
  long step = 0;
  real last_force = 0.0;         // f_x of the last step

  explicit Solver(const oracle_config& cfg) : c(cfg) {
    n[0] = c.nx;
    n[1] = c.ny;
    n[2] = c.nz;
    for (int d = 0; d < 3; ++d) pn[d] = n[d] + 2 * G;
    const double L[3] = {c.lx, c.ly, c.lz};
    for (int d = 0; d < 3; ++d) width[d].assign(pn[d], L[d] / n[d]);
    if (c.y_stretch) {
      // Sec. 3.3: y = tanh(b_g (eta/(1.5 pi) - 1)) / tanh(b_g), eta uniform in [0, 3 pi]:
      // the channel of height 2 (ly = 2 whenever y_stretch is set).
      std::vector<double> yf(c.ny + 1);
      for (int j = 0; j <= c.ny; ++j) {
        const double eta = 3.0 * kPi * j / c.ny;
        yf[j] = std::tanh(c.stretch_b * (eta / (1.5 * kPi) - 1.0)) / std::tanh(c.stretch_b);
      }
      for (int j = 0; j < c.ny; ++j) width[1][j + G] = yf[j + 1] - yf[j];
      for (int m = 0; m < G; ++m) {
        if (c.bc_y == 1) {  // mirror images across the walls
          width[1][G - 1 - m] = width[1][G + m];
          width[1][G + c.ny + m] = width[1][G + c.ny - 1 - m];
        } else {            // periodic images
          width[1][G - 1 - m] = width[1][G + c.ny - 1 - m];
          width[1][G + c.ny + m] = width[1][G + m];
        }
      }
    }
    q.assign(size_t(5) * pn[0] * pn[1] * pn[2], 0.0);
  }

  size_t cells_padded() const { return size_t(pn[0]) * pn[1] * pn[2]; }
  size_t at(int i, int j, int k) const {
    return (size_t(k + G) * pn[1] + (j + G)) * pn[0] + (i + G);
  }
  real& Q(std::vector<real>& a, int v, int i, int j, int k) {
    return a[v * cells_padded() + at(i, j, k)];
  }
  double w(int d, int idx) const { return width[d][idx + G]; }

  // Ghost-cell fill, axes in the order x, y, z so that edges and corners take
  // their values from layers that are already filled.
  void fill_ghosts(std::vector<real>& a) {
    // x: periodic
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int m = 1; m <= G; ++m)
          for (int v = 0; v < 5; ++v) {
            Q(a, v, -m, j, k) = Q(a, v, n[0] - m, j, k);
            Q(a, v, n[0] - 1 + m, j, k) = Q(a, v, m - 1, j, k);
          }
    // y: periodic, or isothermal no-slip walls (Sec. 3.3).
    for (int k = 0; k < n[2]; ++k)
      for (int i = -G; i < n[0] + G; ++i)
        for (int m = 1; m <= G; ++m) {
          if (c.bc_y == 0) {
            for (int v = 0; v < 5; ++v) {
              Q(a, v, i, -m, k) = Q(a, v, i, n[1] - m, k);
              Q(a, v, i, n[1] - 1 + m, k) = Q(a, v, i, m - 1, k);
            }
          } else {
            wall_ghost(a, i, m - 1, -m, k);
            wall_ghost(a, i, n[1] - m, n[1] - 1 + m, k);
          }
        }
    // z: periodic
    for (int j = -G; j < n[1] + G; ++j)
      for (int i = -G; i < n[0] + G; ++i)
        for (int m = 1; m <= G; ++m)
          for (int v = 0; v < 5; ++v) {
            Q(a, v, i, j, -m) = Q(a, v, i, j, n[2] - m);
            Q(a, v, i, j, n[2] - 1 + m) = Q(a, v, i, j, m - 1);
          }
  }

  // Reading (Sec. 3.3 names the isothermal no-slip wall but not its ghost
  // cells): the ghost cell mirrors interior cell jm with velocity negated,
  // equal pressure and temperature T_g = 2 T_wall - T_m (floored at T_wall/2),
  // so that the face average of u and of T equals the wall values.
  void wall_ghost(std::vector<real>& a, int i, int jm, int jg, int k) {
    const double g1 = c.gamma - 1.0;
    const real rho = Q(a, 0, i, jm, k);
    const real u = Q(a, 1, i, jm, k) / rho, v = Q(a, 2, i, jm, k) / rho,
                 ww = Q(a, 3, i, jm, k) / rho;
    const real p = g1 * (Q(a, 4, i, jm, k) - 0.5 * rho * (u * u + v * v + ww * ww));
    real Tg = 2.0 * c.T_wall - p / rho;
    if (Tg < 0.5 * c.T_wall) Tg = 0.5 * c.T_wall;
    const real rg = p / Tg;
    Q(a, 0, i, jg, k) = rg;
    Q(a, 1, i, jg, k) = -rg * u;
    Q(a, 2, i, jg, k) = -rg * v;
    Q(a, 3, i, jg, k) = -rg * ww;
    Q(a, 4, i, jg, k) = p / g1 + 0.5 * rg * (u * u + v * v + ww * ww);
  }

  // Padded index of the cell with coordinate nn along d, aa along t1, bb along t2,
  // where (d, t1, t2) is a cyclic permutation of (x, y, z).
  size_t cell(int d, int nn, int aa, int bb) const {
    int x[3];
    x[d] = nn;
    x[(d + 1) % 3] = aa;
    x[(d + 2) % 3] = bb;
    return at(x[0], x[1], x[2]);
  }
  // Conservative state of a cell in the local frame of direction d:
  // (rho, rho u_n, rho u_t1, rho u_t2, rho E).
  void local(const std::vector<real>& a, int d, size_t ci, real out[5]) const {
    const size_t S = cells_padded();
    out[0] = a[ci];
    out[1] = a[(1 + d) * S + ci];
    out[2] = a[(1 + (d + 1) % 3) * S + ci];
    out[3] = a[(1 + (d + 2) % 3) * S + ci];
    out[4] = a[4 * S + ci];
  }

  // Fluxes through all faces normal to d: Fd[((f * nt1) + a) * nt2 + b][10],
  // f = 0..n_d (face f lies between cells f-1 and f), F then dF, global frame.
  void direction_fluxes(const std::vector<real>& a, int d, double dt, std::vector<real>& Fd) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int nd = n[d], na = n[t1], nb = n[t2];
    const int ea = na + 4, eb = nb + 4;  // face fields carry 2 tangential ghost rows
    const int mode = c.recon;
    // Face fields, local frame: 0 Q_l, 1 Q_r, 2 dQ_l/dn, 3 dQ_r/dn, 4 Q0,
    // 5 dQ0/dn, 6 Qm = the mean of the two cell averages beside the face.
    constexpr int NF = 35;
    std::vector<real> FF(size_t(nd + 1) * ea * eb * NF);
    // Reading: with characteristic reconstruction every reconstruction that
    // serves face point P (the normal one at P, the t1 pass centred at P and
    // the t2 pass of P's Gauss points) uses the eigenvectors of the Euler
    // Jacobian along the face normal at Qm of P.
    const bool chr = c.char_recon != 0;
#pragma omp parallel for collapse(2) schedule(static)
    for (int f = 0; f <= nd; ++f)
      for (int aa = -2; aa < na + 2; ++aa)
        for (int bb = -2; bb < nb + 2; ++bb) {
          // Cell averages of cells f-3 .. f+2 along the normal.
          real qc[6][5];
          for (int s = 0; s < 6; ++s) local(a, d, cell(d, f - 3 + s, aa, bb), qc[s]);
          const double hl = w(d, f - 1), hr = w(d, f);
          real* out = &FF[((size_t(f) * ea + (aa + 2)) * eb + (bb + 2)) * NF];
          for (int v = 0; v < 5; ++v) out[30 + v] = 0.5 * (qc[2][v] + qc[3][v]);
          CharBasis B;
          if (chr) B = char_basis(&out[30], c.gamma);
          real e[4][5];
          normal_end_values(qc, mode, chr ? &B : nullptr, e);
          for (int v = 0; v < 5; ++v) {
            const real QRi = e[0][v], QLi = e[1][v], QLr = e[2][v], QRr = e[3][v];
            out[0 * 5 + v] = QRi;  // Q_l at the face
            out[1 * 5 + v] = QLr;  // Q_r at the face
            // Reading: normal slopes of the quadratic through both end values
            // and the average of the cell (the Remark-1 quadratic, applied in
            // the normal direction), evaluated at the face.
            out[2 * 5 + v] = (4.0 * QRi + 2.0 * QLi - 6.0 * qc[2][v]) / hl;
            out[3 * 5 + v] = -(4.0 * QLr + 2.0 * QRr - 6.0 * qc[3][v]) / hr;
            // Reading: equilibrium slope = derivative at the face of the cubic
            // whose averages over cells i-1 .. i+2 equal the data.
            out[5 * 5 + v] =
                (qc[1][v] - 15.0 * qc[2][v] + 15.0 * qc[3][v] - qc[4][v]) / (6.0 * (hl + hr));
          }
          // Q0 by the compatibility condition: int_{u>0} psi g_l + int_{u<0} psi g_r.
          const Maxwellian gl = maxwellian(&out[0], c.gamma);
          const Maxwellian gr = maxwellian(&out[5], c.gamma);
          for (int i = 0; i < 5; ++i) {
            const Poly pi = psi(i);
            out[4 * 5 + i] = gl.rho * mom(gl, +1, pi) + gr.rho * mom(gr, -1, pi);
          }
        }
    auto ffield = [&](int f, int aa, int bb, int fld) {
      return &FF[((size_t(f) * ea + (aa + 2)) * eb + (bb + 2)) * NF + fld * 5];
    };
    // Tangential reconstruction to the 2x2 Gauss points and the flux there.
    Fd.assign(size_t(nd + 1) * na * nb * 10, 0.0);
#pragma omp parallel for collapse(2) schedule(static)
    for (int f = 0; f <= nd; ++f)
      for (int aa = 0; aa < na; ++aa)
        for (int bb = 0; bb < nb; ++bb) {
          const double h1 = w(t1, aa), h2 = w(t2, bb);
          // t1 pass over rows bb-2 .. bb+2: value and t1-derivative of every
          // field at the two t1 Gauss abscissae.
          real v1[6][5][5][2], d1[6][5][5][2];  // [field][var][row][m]
          for (int r = 0; r < 5; ++r) {
            CharBasis B;
            if (chr) B = char_basis(ffield(f, aa, bb - 2 + r, 6), c.gamma);
            for (int fld = 0; fld < 6; ++fld) {
              real col[5][5], val[2][5], der[2][5];
              for (int s = 0; s < 5; ++s)
                for (int v = 0; v < 5; ++v) col[s][v] = ffield(f, aa - 2 + s, bb - 2 + r, fld)[v];
              tangential_vec(col, mode, chr ? &B : nullptr, val, der);
              for (int v = 0; v < 5; ++v)
                for (int m = 0; m < 2; ++m) {
                  v1[fld][v][r][m] = val[m][v];
                  d1[fld][v][r][m] = der[m][v];
                }
            }
          }
          CharBasis B2;
          if (chr) B2 = char_basis(ffield(f, aa, bb, 6), c.gamma);
          const CharBasis* pb = chr ? &B2 : nullptr;
          real Fsum[10] = {0};
          for (int m = 0; m < 2; ++m)
            for (int mm = 0; mm < 2; ++mm) {
              PointData pd;
              const int vf[3] = {0, 1, 4}, sf[3] = {2, 3, 5};
              for (int s = 0; s < 3; ++s) {
                real col[5][5], val[2][5], der[2][5];
                for (int r = 0; r < 5; ++r)
                  for (int v = 0; v < 5; ++v) col[r][v] = v1[vf[s]][v][r][m];
                tangential_vec(col, mode, pb, val, der);
                for (int v = 0; v < 5; ++v) {
                  pd.st[s][0][v] = val[mm][v];       // value
                  pd.st[s][3][v] = der[mm][v] / h2;  // d/dt2
                }
                for (int r = 0; r < 5; ++r)
                  for (int v = 0; v < 5; ++v) col[r][v] = d1[vf[s]][v][r][m];
                tangential_vec(col, mode, pb, val, der);
                for (int v = 0; v < 5; ++v) pd.st[s][2][v] = val[mm][v] / h1;  // d/dt1
                for (int r = 0; r < 5; ++r)
                  for (int v = 0; v < 5; ++v) col[r][v] = v1[sf[s]][v][r][m];
                tangential_vec(col, mode, pb, val, der);
                for (int v = 0; v < 5; ++v) pd.st[s][1][v] = val[mm][v];  // d/dn
              }
              real F[5], dF[5];
              flux_point(c, pd, dt, F, dF);
              for (int i = 0; i < 5; ++i) {
                Fsum[i] += 0.25 * F[i];  // Gauss weights omega_mn = 1/4 of the face
                Fsum[5 + i] += 0.25 * dF[i];
              }
            }
          // Back to the global frame.
          real* out = &Fd[((size_t(f) * na + aa) * nb + bb) * 10];
          for (int s = 0; s < 2; ++s) {
            const real* L = &Fsum[5 * s];
            real* o = &out[5 * s];
            o[0] = L[0];
            o[1 + d] = L[1];
            o[1 + t1] = L[2];
            o[1 + t2] = L[3];
            o[4] = L[4];
          }
        }
  }

  // L(Q) and dL(Q)/dt on interior cells (Eq. (4)): -(1/|Omega|) sum of the
  // six face fluxes; with face area / cell volume = 1 / (cell width along d).
  // Per cell the faces are taken in the order x-, x+, y-, y+, z-, z+.
  void rhs(std::vector<real>& a, double dt, std::vector<real>& L, std::vector<real>& dL) {
    fill_ghosts(a);
    std::vector<real> Fd[3];
    for (int d = 0; d < 3; ++d) direction_fluxes(a, d, dt, Fd[d]);
    const size_t N = size_t(n[0]) * n[1] * n[2];
    L.assign(5 * N, 0.0);
    dL.assign(5 * N, 0.0);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          const int x[3] = {i, j, k};
          const size_t ci = (size_t(k) * n[1] + j) * n[0] + i;
          real acc[10] = {0};
          for (int d = 0; d < 3; ++d) {
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            const int na = n[t1], nb = n[t2];
            const real* Fm = &Fd[d][((size_t(x[d]) * na + x[t1]) * nb + x[t2]) * 10];
            const real* Fp = &Fd[d][((size_t(x[d] + 1) * na + x[t1]) * nb + x[t2]) * 10];
            const double hd = w(d, x[d]);
            for (int s = 0; s < 10; ++s) acc[s] += -Fm[s] / hd + Fp[s] / hd;
          }
          for (int v = 0; v < 5; ++v) {
            L[v * N + ci] = -acc[v];
            dL[v * N + ci] = -acc[5 + v];
          }
        }
  }

  real cfl_dt() {
    const double g1 = c.gamma - 1.0;
    real best = 1e300;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          const real rho = Q(q, 0, i, j, k);
          const real u[3] = {Q(q, 1, i, j, k) / rho, Q(q, 2, i, j, k) / rho,
                               Q(q, 3, i, j, k) / rho};
          const real p = g1 * (Q(q, 4, i, j, k) - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
          const real cs = sqrt(c.gamma * p / rho);
          const int x[3] = {i, j, k};
          for (int d = 0; d < 3; ++d) {
            const real v = w(d, x[d]) / (fabs(u[d]) + cs);
            if (v < best) best = v;
          }
        }
    return c.cfl * best;
  }

  // One S2O4 step (Eq. (6)), then the streamwise body force of Sec. 3.3.
  double do_step(double dt) {
    if (dt <= 0.0) dt = value(cfl_dt());
    const size_t N = size_t(n[0]) * n[1] * n[2];
    std::vector<real> L0, dL0, L1, dL1;
    std::vector<real> qs = q;  // Q*
    rhs(q, dt, L0, dL0);
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            const size_t ci = (size_t(k) * n[1] + j) * n[0] + i;
            Q(qs, v, i, j, k) = s2o4_stage1(Q(q, v, i, j, k), L0[v * N + ci], dL0[v * N + ci], dt);
          }
    rhs(qs, dt, L1, dL1);
    // Second stage without the force: Q~^{n+1}.
    std::vector<real> qn = q;
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            const size_t ci = (size_t(k) * n[1] + j) * n[0] + i;
            Q(q, v, i, j, k) = s2o4_stage2(Q(qn, v, i, j, k), L0[v * N + ci], dL0[v * N + ci],
                                           dL1[v * N + ci], dt);
          }
    // Streamwise force of Sec. 3.3.  force_mode 0: the constant f_x.
    // force_mode 1: f_x = (int rho U_b - int (rho U)~^{n+1}) /
    // (dt * 1/2 int (rho^n + rho~^{n+1})), which makes int (rho U)^{n+1} equal
    // the target; int rho U_b is read as mass_flux times the box volume.
    real f = c.force_x;
    if (c.force_mode == 1) {
      double vol = 0.0;
      real mom = 0.0, half_rho = 0.0;
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            const double dv = w(0, i) * w(1, j) * w(2, k);
            vol += dv;
            mom += Q(q, 1, i, j, k) * dv;
            half_rho += 0.5 * (Q(qn, 0, i, j, k) + Q(q, 0, i, j, k)) * dv;
          }
      f = (c.mass_flux * vol - mom) / (dt * half_rho);
    }
    last_force = f;
    if (f != 0.0) {
      // (rho U)^{n+1} = (rho U)~ + dt/2 (rho^{n+1} + rho^n) f_x,
      // (rho E)^{n+1} = (rho E)~ + dt/2 ((rho U)^{n+1} + (rho U)^n) f_x.
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            Q(q, 1, i, j, k) += 0.5 * dt * (Q(q, 0, i, j, k) + Q(qn, 0, i, j, k)) * f;
            Q(q, 4, i, j, k) += 0.5 * dt * (Q(q, 1, i, j, k) + Q(qn, 1, i, j, k)) * f;
          }
    }
    t += dt;
    ++step;
    return dt;
  }
};

}  // namespace

extern "C" {

// Threads the oracle's parallel loops use (OpenMP's maximum; 1 without OpenMP).
int oracle_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void* oracle_create(const oracle_config* cfg) { return new Solver(*cfg); }
void oracle_destroy(void* h) { delete static_cast<Solver*>(h); }

// Conservative cell averages in/out, FP64 [5][nz][ny][nx].
void oracle_set_state(void* h, const double* cons) {
  Solver& s = *static_cast<Solver*>(h);
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i)
          s.Q(s.q, v, i, j, k) = cons[((size_t(v) * s.n[2] + k) * s.n[1] + j) * s.n[0] + i];
}
void oracle_get_state(void* h, double* cons) {
  Solver& s = *static_cast<Solver*>(h);
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i)
          cons[((size_t(v) * s.n[2] + k) * s.n[1] + j) * s.n[0] + i] = value(s.Q(s.q, v, i, j, k));
}
// Advance nsteps; dt <= 0 takes the CFL step each time.  Returns the last dt.
double oracle_step(void* h, int nsteps, double dt) {
  Solver& s = *static_cast<Solver*>(h);
  double used = 0.0;
  for (int n = 0; n < nsteps; ++n) used = s.do_step(dt);
  return used;
}
double oracle_time(void* h) { return static_cast<Solver*>(h)->t; }
// Streamwise force f_x applied in the last step.
double oracle_last_force(void* h) { return value(static_cast<Solver*>(h)->last_force); }
double oracle_cfl_dt(void* h) { return value(static_cast<Solver*>(h)->cfl_dt()); }

#ifdef ORACLE_COUNT
// Counting build only: the tallies since the last reset, out[7] = additions
// and subtractions, multiplications, divisions, sqrt, exp, erfc, pow calls.
void oracle_count_get(unsigned long long* out) {
  const oracle_count::Tally& t = oracle_count::g_tally;
  const unsigned long long v[7] = {t.add, t.mul, t.div, t.sqrt, t.exp, t.erfc, t.pow};
  for (int i = 0; i < 7; ++i) out[i] = v[i];
}
void oracle_count_reset() { oracle_count::g_tally = oracle_count::Tally{}; }
#endif

#ifdef ORACLE_TANGENT
// Tangent build only: the derivative part of the state.  oracle_set_state
// sets the values with a zero tangent; oracle_set_tangent then sets the
// direction dQ^0, and after oracle_step (with a fixed dt > 0)
// oracle_get_tangent returns dQ^n = (dQ^n/dQ^0) dQ^0, [5][nz][ny][nx].
void oracle_set_tangent(void* h, const double* dcons) {
  Solver& s = *static_cast<Solver*>(h);
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i)
          s.Q(s.q, v, i, j, k).d = dcons[((size_t(v) * s.n[2] + k) * s.n[1] + j) * s.n[0] + i];
}
void oracle_get_tangent(void* h, double* dcons) {
  Solver& s = *static_cast<Solver*>(h);
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i)
          dcons[((size_t(v) * s.n[2] + k) * s.n[1] + j) * s.n[0] + i] =
              oracle_dual::tangent(s.Q(s.q, v, i, j, k));
}
#endif  // ORACLE_TANGENT

#if !defined(ORACLE_TANGENT) && !defined(ORACLE_COUNT)
// Characteristic basis at the local-frame state Qm: R and R^{-1}, row-major.
void oracle_char_basis(const double* Qm, double gamma, double* R, double* L) {
  const CharBasis B = char_basis(Qm, gamma);
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      R[i * 5 + k] = B.R[i][k];
      L[i * 5 + k] = B.L[i][k];
    }
}
// Normal WENO5 end values of the two cells beside a face from six cell
// averages qc[6][5] (local frame): out[4][5] as normal_end_values; use_char
// selects the characteristic variables of the mean of qc[2] and qc[3].
void oracle_normal_end_values(const double* qc, int mode, int use_char, double gamma, double* out) {
  double q[6][5], e[4][5], qm[5];
  for (int s = 0; s < 6; ++s)
    for (int i = 0; i < 5; ++i) q[s][i] = qc[s * 5 + i];
  for (int i = 0; i < 5; ++i) qm[i] = 0.5 * (q[2][i] + q[3][i]);
  const CharBasis B = char_basis(qm, gamma);
  normal_end_values(q, mode, use_char ? &B : nullptr, e);
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 5; ++i) out[k * 5 + i] = e[k][i];
}
// Tangential reconstruction of a 5-vector field from five face averages
// f[5][5]: values and derivatives at the two Gauss abscissae, out[2][5] each;
// use_char selects the characteristic variables of Qm.
void oracle_tangential_vec(const double* f, int mode, int use_char, const double* Qm, double gamma,
                           double* val, double* der) {
  double F[5][5], v[2][5], d[2][5];
  for (int s = 0; s < 5; ++s)
    for (int i = 0; i < 5; ++i) F[s][i] = f[s * 5 + i];
  const CharBasis B = char_basis(Qm, gamma);
  tangential_vec(F, mode, use_char ? &B : nullptr, v, d);
  for (int m = 0; m < 2; ++m)
    for (int i = 0; i < 5; ++i) {
      val[m * 5 + i] = v[m][i];
      der[m * 5 + i] = d[m][i];
    }
}
// L(Q) and dL/dt of the current state (interior cells, [5][nz][ny][nx]).
void oracle_rhs(void* h, double dt, double* L, double* dL) {
  Solver& s = *static_cast<Solver*>(h);
  std::vector<double> a = s.q, l, dl;
  s.rhs(a, dt, l, dl);
  std::memcpy(L, l.data(), l.size() * sizeof(double));
  std::memcpy(dL, dl.data(), dl.size() * sizeof(double));
}
// Cell widths along axis d for the interior cells.
void oracle_widths(void* h, int d, double* out) {
  Solver& s = *static_cast<Solver*>(h);
  for (int i = 0; i < s.n[d]; ++i) out[i] = s.w(d, i);
}
// Padded state after the ghost fill, [5][nz+6][ny+6][nx+6].
void oracle_padded(void* h, double* out) {
  Solver& s = *static_cast<Solver*>(h);
  std::vector<double> a = s.q;
  s.fill_ghosts(a);
  std::memcpy(out, a.data(), a.size() * sizeof(double));
}

// ---- single pieces, for the pins in tests/ ----

// Normalised moments of the Maxwellian (U, V, W, lambda): uf/up/un/v/w[0..9], xi[0..3].
void oracle_moments(double U, double V, double W, double lam, double K, double* uf, double* up,
                    double* un, double* v, double* w, double* xi) {
  Maxwellian g;
  g.rho = 1.0;
  g.U = U;
  g.V = V;
  g.W = W;
  g.lam = lam;
  set_moments(g, K);
  for (int n = 0; n < kMaxDeg; ++n) {
    uf[n] = g.uf[n];
    up[n] = g.up[n];
    un[n] = g.un[n];
    v[n] = g.v[n];
    w[n] = g.w[n];
  }
  for (int m = 0; m < 4; ++m) xi[m] = g.xi[m];
}
// Slope solve M(Q) a = b for the conservative state Q.
void oracle_slope(const double* Q, double gamma, const double* b, double* a) {
  const Maxwellian g = maxwellian(Q, gamma);
  slope_solve(g, b, a);
}
// Slopes a[3][5] and time coefficient A[5] of a state with derivatives dQ[3][5].
void oracle_kinetic(const double* Q, const double* dQ, double gamma, double* a, double* A) {
  double d[3][5];
  for (int s = 0; s < 3; ++s)
    for (int i = 0; i < 5; ++i) d[s][i] = dQ[s * 5 + i];
  const Kin k = kinetic(Q, d, gamma);
  for (int s = 0; s < 3; ++s)
    for (int i = 0; i < 5; ++i) a[s * 5 + i] = k.a[s][i];
  for (int i = 0; i < 5; ++i) A[i] = k.A[i];
}
// Equilibrium Q0 of the compatibility condition for left / right states.
void oracle_compat(const double* Ql, const double* Qr, double gamma, double* Q0) {
  const Maxwellian gl = maxwellian(Ql, gamma), gr = maxwellian(Qr, gamma);
  for (int i = 0; i < 5; ++i) {
    const Poly pi = psi(i);
    Q0[i] = gl.rho * mom(gl, +1, pi) + gr.rho * mom(gr, -1, pi);
  }
}
void oracle_time_integrals(double T, double tau, double* q) { time_integrals(T, tau, q); }
double oracle_s2o4_stage1(double Qn, double L0, double dL0, double dt) {
  return s2o4_stage1(Qn, L0, dL0, dt);
}
double oracle_s2o4_stage2(double Qn, double L0, double dL0, double dL1, double dt) {
  return s2o4_stage2(Qn, L0, dL0, dL1, dt);
}
double oracle_weno5_right(const double* q, int mode) { return weno5_right(q, mode); }
double oracle_weno5_left(const double* q, int mode) { return weno5_left(q, mode); }
void oracle_tangential(const double* f, int mode, double* val, double* der) {
  tangential(f, mode, val, der);
}
// Flux at one Gauss point; st is [3][4][5]: states l, r, 0 with value and
// derivatives along n, t1, t2, local frame.
void oracle_flux_point(const oracle_config* cfg, const double* st, double dt, double* F,
                       double* dF) {
  PointData pd;
  std::memcpy(pd.st, st, sizeof(pd.st));
  flux_point(*cfg, pd, dt, F, dF);
}

#endif  // the plain build

}  // extern "C"

// Host check of the reverse-mode flux derivatives (flux_rev.cuh) against
// forward-mode dual numbers through the forward functions (physics.cuh), on
// seeded states in double precision, with the constant and the power-law
// viscosity: the cotangents of values AND slopes of the full flux
// (flux_full_vjp, all three states), of its equilibrium and half-space parts
// (with their tau-weighted moment sums), of the smooth flux with and without
// F, and of the compatibility state's sign moments.  Prints the largest
// relative difference over the trials.
// Test support: built and run by tests/test_flux_vjp.py; not part of the
// library.
#include <cmath>
#include <cstdio>
#include <random>

#include "dual.cuh"
#include "flux_rev.cuh"

using namespace hgks;
using D = Dual<double>;

namespace {

double worst = 0.0;

void record(double rev, double fwd, double scale) {
  const double err = std::fabs(rev - fwd) / (scale > 0 ? scale : 1.0);
  if (err > worst) worst = err;
}

// Dual copy of st with a unit tangent on input component c (0-4: q, 5-19: dq[d][i] at 5 + 5 d + i).
PointState<D> seed(const PointState<double>& st, int c) {
  PointState<D> x;
  for (int i = 0; i < 5; ++i) {
    x.q[i] = D(st.q[i], c == i ? 1.0 : 0.0);
    for (int d = 0; d < 3; ++d) x.dq[d][i] = D(st.dq[d][i], c == 5 + 5 * d + i ? 1.0 : 0.0);
  }
  return x;
}

double component(const PointState<double>& cot, int c) {
  return c < 5 ? cot.q[c] : cot.dq[(c - 5) / 5][(c - 5) % 5];
}

void zero(PointState<double>& p) {
  for (int i = 0; i < 5; ++i) {
    p.q[i] = 0.0;
    for (int d = 0; d < 3; ++d) p.dq[d][i] = 0.0;
  }
}

PointState<double> random_state(std::mt19937_64& rng, const Gas<double>& g, double vel) {
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  PointState<double> st;
  st.q[0] = 0.3 * u(rng);
  st.q[1] = vel * u(rng);
  st.q[2] = vel * u(rng);
  st.q[3] = vel * u(rng);
  st.q[4] = 0.3 * g.p_r / g.gm1 * u(rng) +
            0.5 * (st.q[1] * st.q[1] + st.q[2] * st.q[2] + st.q[3] * st.q[3]) / (g.rho_r + st.q[0]);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 5; ++i) st.dq[d][i] = (i == 4 ? g.p_r : 1.0) * u(rng);
  return st;
}

}  // namespace

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  for (int trial = 0; trial < 200; ++trial) {
    Gas<double> g;
    g.gamma = 1.4;
    g.gm1 = 0.4;
    g.K = (5.0 - 3.0 * 1.4) / 0.4;
    g.pr_fix = 1.0 / 0.72 - 1.0;
    g.visc_law = trial % 2;
    g.mu_ref = 1e-3;
    g.T_ref_inv = 1.0;
    g.visc_exp = 0.76;
    g.tau_num_C = 1.0;
    g.rho_r = 1.0;
    g.p_r = trial % 3 == 0 ? 71.43 : 1.0;
    g.h_r = g.gamma / g.gm1 * g.p_r;
    const Gas<D> gd = dual_gas(g);
    const double vel = trial % 3 == 0 ? 3.0 : 0.8;
    const PointState<double> st = random_state(rng, g, vel);
    // Fit weights (dual numbers in tau) and flux cotangents; gV, Gt the
    // cotangents of the moment vectors and their tau derivatives.
    double wF[5], wdF[5];
    D Fq[3], dFq[3];
    for (int i = 0; i < 5; ++i) {
      wF[i] = u(rng);
      wdF[i] = u(rng);
    }
    for (int k = 0; k < 3; ++k) {
      Fq[k] = D(u(rng), u(rng));
      dFq[k] = D(u(rng), u(rng));
    }
    double gV[3][5], Gt[3][5];
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 5; ++i) {
        gV[k][i] = wF[i] * Fq[k].v + wdF[i] * dFq[k].v;
        Gt[k][i] = wF[i] * Fq[k].d + wdF[i] * dFq[k].d;
      }
    // Equilibrium part: J = gV . V - wpr tau p0 dT0 (tau fixed); phi = Gt . V - wpr p0 dT0.
    {
      const double wpr = u(rng), tau = 0.01 * (1.5 + u(rng));
      PointState<double> cot;
      zero(cot);
      const double phi = flux_full_eq_rev(st, g, wF, wdF, Fq, dFq, wpr, tau, cot);
      FullEq<double> e0;
      flux_full_eq(st, g, e0);
      double phi_ref = -wpr * e0.p * e0.dT, phi_scale = std::fabs(phi_ref);
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 5; ++i) {
          phi_ref += Gt[k][i] * e0.V[k][i];
          phi_scale += std::fabs(Gt[k][i] * e0.V[k][i]);
        }
      record(phi, phi_ref, phi_scale);
      for (int c = 0; c < 20; ++c) {
        FullEq<D> e;
        flux_full_eq(seed(st, c), gd, e);
        const double pr_term = -wpr * tau * (e.p * e.dT).d;
        double fwd = pr_term, scale = std::fabs(pr_term);
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 5; ++i) {
            fwd += gV[k][i] * e.V[k][i].d;
            scale += std::fabs(gV[k][i] * e.V[k][i].d);
          }
        record(component(cot, c), fwd, scale);
      }
    }
    // Half-space parts: J = gV . V; phi = Gt . V.
    for (int side = 0; side < 2; ++side) {
      PointState<double> cot;
      zero(cot);
      const double phi = flux_full_side_rev(st, g, side, wF, wdF, Fq, dFq, cot);
      FullSide<double> h0;
      flux_full_side(st, g, side, h0);
      double phi_ref = 0.0, phi_scale = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 5; ++i) {
          phi_ref += Gt[k][i] * h0.V[k][i];
          phi_scale += std::fabs(Gt[k][i] * h0.V[k][i]);
        }
      record(phi, phi_ref, phi_scale);
      for (int c = 0; c < 20; ++c) {
        FullSide<D> h;
        flux_full_side(seed(st, c), gd, side, h);
        double fwd = 0.0, scale = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 5; ++i) {
            fwd += gV[k][i] * h.V[k][i].d;
            scale += std::fabs(gV[k][i] * h.V[k][i].d);
          }
        record(component(cot, c), fwd, scale);
      }
    }
    // Full flux: J = gF . F + gdF . dF over the three states.
    {
      PointState<double> s3[3] = {st, random_state(rng, g, vel), random_state(rng, g, vel)};
      const double dt = 0.02 * (1.5 + u(rng));
      double gF[5], gdF[5];
      for (int i = 0; i < 5; ++i) {
        gF[i] = u(rng);
        gdF[i] = u(rng);
      }
      PointState<double> cot[3];
      for (int k = 0; k < 3; ++k) zero(cot[k]);
      flux_full_vjp(s3, g, dt, gF, gdF, cot);
      for (int which = 0; which < 3; ++which)
        for (int c = 0; c < 20; ++c) {
          PointState<D> x[3];
          for (int k = 0; k < 3; ++k) x[k] = seed(s3[k], k == which ? c : -1);
          D F[5], dF[5];
          flux_full(x[0], x[1], x[2], gd, D(dt), F, dF);
          double fwd = 0.0, scale = 0.0;
          for (int i = 0; i < 5; ++i) {
            fwd += gF[i] * F[i].d + gdF[i] * dF[i].d;
            scale += std::fabs(gF[i] * F[i].d) + std::fabs(gdF[i] * dF[i].d);
          }
          record(component(cot[which], c), fwd, scale);
        }
    }
    // Sign moments of the compatibility state.
    {
      double gS[5];
      for (int i = 0; i < 5; ++i) gS[i] = u(rng);
      double rev[5] = {0, 0, 0, 0, 0};
      sign_moments_rev(st.q, g, gS, rev);
      for (int c = 0; c < 5; ++c) {
        D x[5], S[5];
        for (int i = 0; i < 5; ++i) x[i] = D(st.q[i], i == c ? 1.0 : 0.0);
        sign_moments(x, gd, S);
        double fwd = 0.0, scale = 0.0;
        for (int i = 0; i < 5; ++i) {
          fwd += gS[i] * S[i].d;
          scale += std::fabs(gS[i] * S[i].d);
        }
        record(rev[c], fwd, scale);
      }
    }
    // Smooth flux, with and without F.
    for (int wantF = 0; wantF < 2; ++wantF) {
      double gF[5], gdF[5];
      for (int i = 0; i < 5; ++i) {
        gF[i] = u(rng);
        gdF[i] = u(rng);
      }
      PointState<double> cot;
      zero(cot);
      flux_smooth_rev(st, g, wantF != 0, gF, gdF, cot);
      for (int c = 0; c < 20; ++c) {
        D F[5], dF[5];
        flux_smooth(seed(st, c), gd, wantF != 0, F, dF);
        double fwd = 0.0, scale = 0.0;
        for (int i = 0; i < 5; ++i) {
          const double a = wantF ? gF[i] * F[i].d : 0.0, b = gdF[i] * dF[i].d;
          fwd += a + b;
          scale += std::fabs(a) + std::fabs(b);
        }
        record(component(cot, c), fwd, scale);
      }
    }
  }
  std::printf("%.3e\n", worst);
  return 0;
}

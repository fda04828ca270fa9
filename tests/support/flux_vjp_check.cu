// Host check of the reverse-mode value cotangents of the fluxes and of the
// compatibility state's sign moments (flux_rev.cuh: the smooth flux, the
// full flux's equilibrium part and both half-space parts, sign_moments)
// against forward-mode dual numbers through the forward functions
// (physics.cuh), on seeded states in double precision, with
// the constant and the power-law viscosity.  Prints the largest relative difference over the trials.
// Test support: built and run by tests/test_flux_vjp.py; not part of the
// library.
#include <cmath>
#include <cstdio>
#include <random>

#include "dual.cuh"
#include "flux_rev.cuh"

using namespace hgks;

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  double worst = 0.0;
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
    PointState<double> st;
    const double vel = trial % 3 == 0 ? 3.0 : 0.8;
    st.q[0] = 0.3 * u(rng);
    st.q[1] = vel * u(rng);
    st.q[2] = vel * u(rng);
    st.q[3] = vel * u(rng);
    st.q[4] = 0.3 * g.p_r / g.gm1 * u(rng) + 0.5 * (st.q[1] * st.q[1] + st.q[2] * st.q[2] + st.q[3] * st.q[3]) /
                                                  (g.rho_r + st.q[0]);
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < 5; ++i) st.dq[d][i] = (i == 4 ? g.p_r : 1.0) * u(rng);
    double gV[3][5], gp = u(rng);
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 5; ++i) gV[k][i] = u(rng);
    // equilibrium part: cotangents of V, mu, p, dT
    {
      const double gmu = u(rng), gp0 = u(rng), gdT = u(rng);
      double rev[5] = {0, 0, 0, 0, 0};
      flux_full_eq_value_rev(st, g, gV, gmu, gp0, gdT, rev);
      const Gas<Dual<double>> gd = dual_gas(g);
      for (int c = 0; c < 5; ++c) {
        PointState<Dual<double>> x;
        for (int i = 0; i < 5; ++i) {
          x.q[i] = Dual<double>(st.q[i], i == c ? 1.0 : 0.0);
          for (int d = 0; d < 3; ++d) x.dq[d][i] = Dual<double>(st.dq[d][i], 0.0);
        }
        FullEq<Dual<double>> e;
        flux_full_eq(x, gd, e);
        double fwd = gmu * e.mu.d + gp0 * e.p.d + gdT * e.dT.d;
        double scale = std::fabs(gmu * e.mu.d) + std::fabs(gp0 * e.p.d) + std::fabs(gdT * e.dT.d);
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 5; ++i) {
            fwd += gV[k][i] * e.V[k][i].d;
            scale += std::fabs(gV[k][i] * e.V[k][i].d);
          }
        const double err = std::fabs(rev[c] - fwd) / (scale > 0 ? scale : 1.0);
        if (err > worst) worst = err;
      }
    }
    // sign moments of the compatibility state
    {
      double gS[5];
      for (int i = 0; i < 5; ++i) gS[i] = u(rng);
      double rev[5] = {0, 0, 0, 0, 0};
      sign_moments_rev(st.q, g, gS, rev);
      const Gas<Dual<double>> gd = dual_gas(g);
      for (int c = 0; c < 5; ++c) {
        Dual<double> x[5], S[5];
        for (int i = 0; i < 5; ++i) x[i] = Dual<double>(st.q[i], i == c ? 1.0 : 0.0);
        sign_moments(x, gd, S);
        double fwd = 0.0, scale = 0.0;
        for (int i = 0; i < 5; ++i) {
          fwd += gS[i] * S[i].d;
          scale += std::fabs(gS[i] * S[i].d);
        }
        const double err = std::fabs(rev[c] - fwd) / (scale > 0 ? scale : 1.0);
        if (err > worst) worst = err;
      }
    }
    // smooth flux, with and without F
    for (int wantF = 0; wantF < 2; ++wantF) {
      double gF[5], gdF[5];
      for (int i = 0; i < 5; ++i) {
        gF[i] = u(rng);
        gdF[i] = u(rng);
      }
      double rev[5] = {0, 0, 0, 0, 0};
      flux_smooth_value_rev(st, g, wantF != 0, gF, gdF, rev);
      const Gas<Dual<double>> gd = dual_gas(g);
      for (int c = 0; c < 5; ++c) {
        PointState<Dual<double>> x;
        for (int i = 0; i < 5; ++i) {
          x.q[i] = Dual<double>(st.q[i], i == c ? 1.0 : 0.0);
          for (int d = 0; d < 3; ++d) x.dq[d][i] = Dual<double>(st.dq[d][i], 0.0);
        }
        Dual<double> F[5], dF[5];
        flux_smooth(x, gd, wantF != 0, F, dF);
        double fwd = 0.0, scale = 0.0;
        for (int i = 0; i < 5; ++i) {
          const double a = wantF ? gF[i] * F[i].d : 0.0, b = gdF[i] * dF[i].d;
          fwd += a + b;
          scale += std::fabs(a) + std::fabs(b);
        }
        const double err = std::fabs(rev[c] - fwd) / (scale > 0 ? scale : 1.0);
        if (err > worst) worst = err;
      }
    }
    for (int side = 0; side < 2; ++side) {
      double rev[5] = {0, 0, 0, 0, 0};
      flux_full_side_value_rev(st, g, side, gV, gp, rev);
      const Gas<Dual<double>> gd = dual_gas(g);
      for (int c = 0; c < 5; ++c) {
        PointState<Dual<double>> x;
        for (int i = 0; i < 5; ++i) {
          x.q[i] = Dual<double>(st.q[i], i == c ? 1.0 : 0.0);
          for (int d = 0; d < 3; ++d) x.dq[d][i] = Dual<double>(st.dq[d][i], 0.0);
        }
        FullSide<Dual<double>> h;
        flux_full_side(x, gd, side, h);
        double fwd = gp * h.p.d;
        double scale = std::fabs(gp * h.p.d);
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 5; ++i) {
            fwd += gV[k][i] * h.V[k][i].d;
            scale += std::fabs(gV[k][i] * h.V[k][i].d);
          }
        const double err = std::fabs(rev[c] - fwd) / (scale > 0 ? scale : 1.0);
        if (err > worst) worst = err;
      }
    }
  }
  std::printf("%.3e\n", worst);
  return 0;
}

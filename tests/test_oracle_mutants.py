"""Planted mistakes in the oracle are caught by its pins (CPU only).

Each case copies oracle/ into a temporary directory, plants one plausible
mistake in the copy's source - the C++ scheme or the numpy statistics: a
swapped index, slot or width, a wrong coefficient, sign or stencil - and runs, against the copy, the pins that
must catch it: at least one has to fail.  The unmodified copy passes the
same pins.  The repository's own oracle is never modified.  A planted
pattern that no longer occurs in the source fails the test, so the list
follows the source.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ANISO = "tests/test_oracle_scheme.py::test_operator_converges_on_an_anisotropic_box"
OBLIQUE = "tests/test_oracle_scheme.py::test_linear_smooth_operator_is_fifth_order_on_oblique_wave"
ASSEMBLY = "tests/test_oracle_assembly.py"
REFLECT = "tests/test_oracle_symmetry.py::test_step_commutes_with_a_reflection"
BRUTE = "tests/test_oracle_flux.py::test_full_flux_matches_brute_force_phase_space_quadrature"
POWER = "tests/test_oracle_flux.py::test_shear_stress_follows_the_power_law_viscosity"
S2O4 = "tests/test_oracle_pieces.py::test_s2o4_on_linear_ode_is_the_fourth_order_taylor_polynomial"
WENOZ = "tests/test_oracle_pieces.py::test_weno_z_is_linear_where_the_outer_indicators_agree"
WENOQ = "tests/test_oracle_pieces.py::test_weno5_exact_on_quadratics"
MOMENTS = "tests/test_oracle_pieces.py::test_moments_match_quadrature"
QUARTIC = "tests/test_oracle_pieces.py::test_tangential_quartic_exact"
WALL = "tests/test_oracle_scheme.py::test_wall_ghost_cells"
WENODEF = "tests/test_oracle_pieces.py::test_weno5_matches_its_definition_on_random_data"
HEAT = "tests/test_oracle_flux.py::test_smooth_flux_heat_flux"
TIMEINT = "tests/test_oracle_pieces.py::test_time_integrals_match_numerical_integration"
TANGQ = "tests/test_oracle_pieces.py::test_tangential_weno_quadratic_exact"
GRID = "tests/test_oracle_scheme.py::test_channel_grid_matches_printed_table"
TGDT = "tests/test_oracle_scheme.py::test_taylor_green_time_steps_match_printed_table"
MASSFLUX = "tests/test_oracle_force.py::test_mass_flux_force_holds_the_target"
ADVECTED = "tests/test_oracle_scheme.py::test_advected_wave_run_converges_at_fifth_order"
FORCE = "tests/test_oracle_force.py::test_constant_force_on_uniform_state_is_exact"
FORCEFORM = ("tests/test_oracle_force.py::"
             "test_mass_flux_force_equals_the_closed_form_and_the_constant_force_step")
WRAP = "tests/test_oracle_scheme.py::test_periodic_ghost_cells_wrap_including_corners"
CHARBASIS = "tests/test_oracle_char.py::test_basis_diagonalises_the_euler_jacobian"
CHARTANG = "tests/test_oracle_char.py::test_tangential_reconstruction_separates_superposed_fields"
CHARNORM = "tests/test_oracle_char.py::test_two_superposed_fields_are_reconstructed_separately"
MOVINGSTRESS = "tests/test_oracle_flux.py::test_normal_stress_work_in_a_moving_gas"
XIMOM = "tests/test_oracle_pieces.py::test_internal_moments_match_radial_quadrature"

# (name, text in hgks_oracle.cpp, planted replacement, pins)
MUTANTS = [
    ("t2 derivative divided by the t1 width",
     "pd.st[s][3][v] = der[mm][v] / h2;", "pd.st[s][3][v] = der[mm][v] / h1;", [ANISO]),
    ("t2 derivative at the t1 Gauss index",
     "pd.st[s][3][v] = der[mm][v] / h2;", "pd.st[s][3][v] = der[m][v] / h2;", [OBLIQUE]),
    ("tangential flux components swapped on output",
     "o[1 + t1] = L[2];\n            o[1 + t2] = L[3];",
     "o[1 + t1] = L[3];\n            o[1 + t2] = L[2];", [ANISO]),
    ("tangential momenta swapped on input",
     "out[2] = a[(1 + (d + 1) % 3) * S + ci];\n    out[3] = a[(1 + (d + 2) % 3) * S + ci];",
     "out[2] = a[(1 + (d + 2) % 3) * S + ci];\n    out[3] = a[(1 + (d + 1) % 3) * S + ci];", [ANISO]),
    ("Gauss weight of dF",
     "Fsum[5 + i] += 0.25 * dF[i];", "Fsum[5 + i] += 0.3 * dF[i];", [OBLIQUE]),
    ("sign of the outer taps of the equilibrium slope",
     "(qc[1][v] - 15.0 * qc[2][v] + 15.0 * qc[3][v] - qc[4][v])",
     "(-qc[1][v] - 15.0 * qc[2][v] + 15.0 * qc[3][v] + qc[4][v])", [OBLIQUE]),
    ("equilibrium slope over the left width only",
     "/ (6.0 * (hl + hr));", "/ (12.0 * hl);", [ASSEMBLY]),
    ("left normal slope over the right width",
     "out[2 * 5 + v] = (4.0 * QRi + 2.0 * QLi - 6.0 * qc[2][v]) / hl;",
     "out[2 * 5 + v] = (4.0 * QRi + 2.0 * QLi - 6.0 * qc[2][v]) / hr;", [ASSEMBLY]),
    ("normal slopes of the left and right states exchanged",
     "sf[3] = {2, 3, 5}", "sf[3] = {3, 2, 5}", [ASSEMBLY]),
    ("Heaviside factor on the wrong state",
     "out[4 * 5 + i] = gl.rho * mom(gl, +1, pi) + gr.rho * mom(gr, -1, pi);",
     "out[4 * 5 + i] = gl.rho * mom(gl, -1, pi) + gr.rho * mom(gr, +1, pi);", [ASSEMBLY]),
    ("characteristic basis at the left cell instead of the mean",
     "out[30 + v] = 0.5 * (qc[2][v] + qc[3][v]);", "out[30 + v] = qc[2][v];", [REFLECT]),
    ("numerical collision time halved",
     "tau += c.tau_num_C * fabs((pl - pr) / (pl + pr)) * dt;",
     "tau += c.tau_num_C * fabs((pl - pr) / (pl + pr)) * dt * 0.5;", [BRUTE]),
    ("viscosity law inverted",
     "pow(T / c.T_ref, c.visc_exp)", "pow(c.T_ref / T, c.visc_exp)", [POWER]),
    ("S2O4 first-stage coefficient",
     "0.125 * dt * dt * dL0", "0.1 * dt * dt * dL0", [S2O4]),
    ("S2O4 second-stage weights exchanged",
     "dt * dt / 6.0 * (dL0 + 2.0 * dL1)", "dt * dt / 6.0 * (2.0 * dL0 + dL1)", [S2O4]),
    ("WENO-Z indicator from the wrong pair",
     "fabs(beta[0] - beta[2])", "fabs(beta[0] - beta[1])", [WENOZ]),
    ("WENO5 middle candidate coefficient",
     "(-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.0", "(-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.5", [WENOQ]),
    ("Gaussian moment recursion index",
     "(n + 1) / (2.0 * lam) * m[n]", "(n + 2) / (2.0 * lam) * m[n]", [MOMENTS]),
    ("quartic cell averages",
     "(std::pow(hi, p + 1) - std::pow(lo, p + 1)) / (p + 1)",
     "(std::pow(hi, p + 1) - std::pow(lo, p + 1)) / (p + 2)", [QUARTIC]),
    ("wall ghost temperature",
     "real Tg = 2.0 * c.T_wall - p / rho;", "real Tg = 1.5 * c.T_wall - 0.5 * p / rho;", [WALL]),
    ("smoothness indicator coefficient",
     "13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1", "13.0 / 12.0 * s1 * s1 + 0.5 * t1 * t1", [WENODEF]),
    ("flux fit of F",
     "F[i] = (4.0 * W[1][i] - W[0][i]) / dt;", "F[i] = (3.0 * W[1][i] - W[0][i]) / dt;", [BRUTE]),
    ("flux fit of dF",
     "dF[i] = 4.0 * (W[0][i] - 2.0 * W[1][i]) / (dt * dt);",
     "dF[i] = 2.0 * (W[0][i] - 2.0 * W[1][i]) / (dt * dt);", [BRUTE]),
    ("Prandtl correction",
     "F[4] += (1.0 / c.prandtl - 1.0) * q;", "F[4] += (c.prandtl - 1.0) * q;", [HEAT]),
    ("time integral of -(tau + t) e^{-t/tau}",
     "q[4] = tau * (T * e - 2.0 * tau * (1.0 - e));", "q[4] = tau * (T * e - tau * (1.0 - e));",
     [TIMEINT]),
    ("tangential quadratic constant term",
     "a = f[2] - c / 12.0;", "a = f[2] - c / 6.0;", [TANGQ]),
    ("tanh mapping offset",
     "(eta / (1.5 * kPi) - 1.0)", "(eta / (1.5 * kPi) - 0.9)", [GRID]),
    ("CFL sound speed",
     "w(d, x[d]) / (fabs(u[d]) + cs)", "w(d, x[d]) / (fabs(u[d]) + 0.9 * cs)", [TGDT]),
    ("mass-flux force",
     "f = (c.mass_flux * vol - mom) / (dt * half_rho);",
     "f = 0.5 * (c.mass_flux * vol - mom) / (dt * half_rho);", [MASSFLUX]),
    ("second stage with the first stage's dL",
     "dL1[v * N + ci], dt);", "dL0[v * N + ci], dt);", [ADVECTED]),
    ("first stage over half the step",
     "L0[v * N + ci], dL0[v * N + ci], dt);\n          }\n    rhs(qs",
     "L0[v * N + ci], dL0[v * N + ci], 0.5 * dt);\n          }\n    rhs(qs", [ADVECTED]),
    ("wall-normal velocity not reversed in the ghost",
     "Q(a, 2, i, jg, k) = -rg * v;", "Q(a, 2, i, jg, k) = rg * v;", [WALL]),
    ("force work from the old momentum only",
     "(Q(q, 1, i, j, k) + Q(qn, 1, i, j, k)) * f", "2.0 * Q(qn, 1, i, j, k) * f", [FORCE]),
    ("mass-flux force over the old density only",
     "half_rho += 0.5 * (Q(qn, 0, i, j, k) + Q(q, 0, i, j, k)) * dv;",
     "half_rho += Q(qn, 0, i, j, k) * dv;", [FORCEFORM]),
    ("periodic ghost from the wrong layer",
     "Q(a, v, i, j, n[2] - 1 + m) = Q(a, v, i, j, m - 1);",
     "Q(a, v, i, j, n[2] - 1 + m) = Q(a, v, i, j, m);", [WRAP]),
    ("eigenvector of u - c",
     "{1.0, u - c, v, w, H - u * c}", "{1.0, u - c, v, w, H - v * c}", [CHARBASIS]),
    ("characteristic derivatives mapped back with R^-1",
     "mat5(B->R, cd[m], der[m]);", "mat5(B->L, cd[m], der[m]);", [CHARTANG]),
    ("opposite end value of the left cell",
     "e[1][i] = weno5_left(sl, mode);", "e[1][i] = weno5_right(sl, mode);", [CHARNORM, ASSEMBLY]),
    ("sign of the time-coefficient condition",
     "rhs[i] = -s;", "rhs[i] = s;", [BRUTE]),
    ("slope condition without the density",
     "b[i] = dQ[d][i] / Q[0];", "b[i] = dQ[d][i];", [BRUTE]),
    ("derivative of the tangential quadratic",
     "der[m] = b + 2.0 * c * s;", "der[m] = b + c * s;", [TANGQ]),
    ("heat polynomial of the Prandtl correction (xi^2 term)",
     "p.add(-0.5 * U, 0, 0, 0, 1);", "p.add(0.5 * U, 0, 0, 0, 1);", [MOVINGSTRESS]),
    ("sign of the exponential term of the u < 0 half-space moment",
     "g.un[1] = g.U * g.un[0] - e;", "g.un[1] = g.U * g.un[0] + e;", [MOMENTS]),
    ("moments of the internal degrees of freedom",
     "g.xi[m - 1] * (K + 2.0 * (m - 1)) / (2.0 * lam)", "g.xi[m - 1] * (K + 2.0 * m) / (2.0 * lam)",
     [XIMOM]),
    ("lambda of the Maxwellian",
     "g.lam = Q[0] / (2.0 * p);", "g.lam = Q[0] / p;", [BRUTE]),
    ("internal degrees of freedom",
     "const double K = (5.0 - 3.0 * gamma) / (gamma - 1.0);",
     "const double K = (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0;", [BRUTE]),
    ("time integral of (t + tau) e^{-t/tau} - tau",
     "q[1] = 2.0 * tau * tau * (1.0 - e) - tau * T * (1.0 + e);",
     "q[1] = 2.0 * tau * tau * (1.0 - e) - tau * T * (1.0 - e);", [TIMEINT]),
    ("Gauss abscissae",
     "const double kGaussS[2] = {-0.5 / std::sqrt(3.0), 0.5 / std::sqrt(3.0)};",
     "const double kGaussS[2] = {-0.3, 0.3};", [QUARTIC]),
    ("periodic x ghost one cell off",
     "Q(a, v, -m, j, k) = Q(a, v, n[0] - m, j, k);", "Q(a, v, -m, j, k) = Q(a, v, n[0] - m - 1, j, k);",
     [WRAP]),
    ("periodic y ghosts all from one row",
     "Q(a, v, i, -m, k) = Q(a, v, i, n[1] - m, k);", "Q(a, v, i, -m, k) = Q(a, v, i, n[1] - 1, k);",
     [WRAP]),
    ("internal-energy factor of a moment product",
     "c * um[a] * g.v[b] * g.w[w] * g.xi[d]", "c * um[a] * g.v[b] * g.w[w] * g.xi[d > 0 ? d - 1 : 0]",
     [BRUTE]),
    ("w factor of a moment product taken from v",
     "c * um[a] * g.v[b] * g.w[w] * g.xi[d]", "c * um[a] * g.v[b] * g.v[w] * g.xi[d]", [BRUTE]),
]


TG = "tests/test_oracle_turbulence.py::test_taylor_green_closed_forms"
ENSTROPHY = "tests/test_oracle_turbulence.py::test_enstrophy_sixth_order_convergence"
COMPRESSION = "tests/test_oracle_turbulence.py::test_compression_wave"
TWOMODES = "tests/test_oracle_turbulence.py::test_skewness_and_flatness_of_two_modes"
POWERNP = "tests/test_oracle_turbulence.py::test_power_law_viscosity_scales_with_temperature"
POISEUILLE = "tests/test_oracle_channel.py::test_poiseuille_statistics_in_closed_form"
POTENTIAL = "tests/test_oracle_turbulence.py::test_potential_flow_closed_forms"
DENSITY = "tests/test_oracle_channel.py::test_wall_and_bulk_densities_with_a_density_profile"
RHO0 = "tests/test_oracle_turbulence.py::test_reference_density_divides_the_normalised_quantities"

TANFD = "tests/test_oracle_tangent.py::test_tangent_equals_central_differences_where_smooth"

# The dual numbers of the tangent build and the numpy statistics:
# (file, name, text, planted replacement, pins)
STAT_MUTANTS = [
    ("__init__.py", "energy of the primitive-to-conservative map",
     "p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)",
     "p / gamma + 0.5 * rho * (u * u + v * v + w * w)", [CHARBASIS, COMPRESSION]),
    ("__init__.py", "momenta of the primitive-to-conservative map exchanged",
     "return np.stack([rho, rho * u, rho * v, rho * w,", "return np.stack([rho, rho * u, rho * w, rho * v,",
     [POTENTIAL]),
    ("tangent.h", "derivative of sqrt",
     "return {s, x.d / (2.0 * s)};", "return {s, x.d / s};", [TANFD]),
    ("tangent.h", "sign of the derivative of erfc",
     "-two_over_sqrt_pi * std::exp", "two_over_sqrt_pi * std::exp", [TANFD]),
    ("tangent.h", "product rule with a dropped term",
     "return {a.v * b.v, a.d * b.v + a.v * b.d};", "return {a.v * b.v, a.d * b.v};", [TANFD]),
    ("tangent.h", "quotient rule sign",
     "return {q, (a.d - q * b.d) / b.v};", "return {q, (a.d + q * b.d) / b.v};", [TANFD]),
    ("tangent.h", "power rule without the exponent",
     "return {p, e * std::pow(x.v, e - 1.0) * x.d};", "return {p, std::pow(x.v, e - 1.0) * x.d};",
     [TANFD]),
    ("turbulence.py", "sixth-order difference coefficient",
     "(45.0 * s(1) - 9.0 * s(2) + s(3))", "(45.0 * s(1) - 8.0 * s(2) + s(3))", [ENSTROPHY]),
    ("turbulence.py", "vorticity component from the wrong gradient",
     "G[2][1] - G[1][2]", "G[2][1] - G[1][1]", [POTENTIAL]),
    ("turbulence.py", "deviatoric part of the strain rate",
     "(theta / 3.0 if i == j else 0.0)", "(theta / 2.0 if i == j else 0.0)", [COMPRESSION]),
    ("turbulence.py", "bulk viscosity",
     "2.0 * N / (3.0 * (N + 3.0)) * mu", "2.0 * N / (3.0 * (N + 2.0)) * mu", [COMPRESSION]),
    ("turbulence.py", "sign of the pressure-dilatation dissipation",
     'out["eps3"] = -avg(p * theta) / rho0', 'out["eps3"] = avg(p * theta) / rho0', [COMPRESSION]),
    ("turbulence.py", "dilatational dissipation factor",
     'out["eps_d"] = 4.0 / 3.0 * avg', 'out["eps_d"] = avg', [COMPRESSION]),
    ("turbulence.py", "eps2 not normalised by the reference density",
     'out["eps2"] = avg(mu_b * theta ** 2) / rho0', 'out["eps2"] = avg(mu_b * theta ** 2)', [RHO0]),
    ("turbulence.py", "enstrophy not normalised by the reference density",
     'out["zeta"] = avg(0.5 * rho * w2) / rho0', 'out["zeta"] = avg(0.5 * rho * w2)', [RHO0]),
    ("turbulence.py", "skewness normalisation",
     "m3[i] / m2[i] ** 1.5", "m3[i] / m2[i] ** 2", [TWOMODES]),
    ("turbulence.py", "viscosity law",
     "mu_ref * (T / T_ref) ** exp", "mu_ref * (T_ref / T) ** exp", [POWERNP]),
    ("channel.py", "upper-wall slope from swapped rows",
     "hi = _wall_slope(dy[-1], dy[-2], Um[-1], Um[-2])",
     "hi = _wall_slope(dy[-1], dy[-2], Um[-2], Um[-1])", [POISEUILLE]),
    ("channel.py", "bulk Reynolds number length",
     'out["Re_b"] = out["U_b"] * 2.0 * H / nu', 'out["Re_b"] = out["U_b"] * H / nu', [POISEUILLE]),
    ("channel.py", "skin-friction dynamic pressure",
     "(0.5 * out[\"rho_b\"] * out[\"U_b\"] ** 2)", "(out[\"rho_b\"] * out[\"U_b\"] ** 2)",
     [POISEUILLE]),
    ("channel.py", "wall density from the lower wall only",
     'out["rho_w"] = 0.5 * (rm[0] + rm[-1])', 'out["rho_w"] = rm[0]', [DENSITY]),
    ("channel.py", "bulk density without the cell heights",
     'out["rho_b"] = (rm * dy).sum() / ly', 'out["rho_b"] = rm.mean()', [DENSITY]),
    ("channel.py", "centreline cubic about the wrong point",
     "faces[j0 + k] - yc, faces[j0 + k + 1] - yc", "faces[j0 + k] - yc, faces[j0 + k + 1] - yc + 0.01",
     [POISEUILLE]),
]


def all_mutants():
    return [("hgks_oracle.cpp", *m) for m in MUTANTS] + STAT_MUTANTS


def copy_oracle(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    return os.path.join(dst, "oracle", "hgks_oracle.cpp")


def run_pins(workdir, pins):
    """pytest of the pins with the oracle package of workdir first on the path."""
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([workdir, ROOT]), OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           *[os.path.join(ROOT, p) for p in pins]]
    return subprocess.run(cmd, cwd=workdir, env=env, capture_output=True, text=True, timeout=900)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    mutants = all_mutants()
    src = {f: open(os.path.join(ROOT, "oracle", f)).read() for f, *_ in mutants}
    missing = [name for f, name, old, _, _ in mutants if src[f].count(old) != 1]
    assert not missing, f"planted patterns not found once in the source: {missing}"

    control = str(tmp_path / "control")
    copy_oracle(control)
    pins = sorted({p for *_, ps in mutants for p in ps})
    r = run_pins(control, pins)
    assert r.returncode == 0, r.stdout[-3000:]

    def one(k):
        f, name, old, new, ps = mutants[k]
        work = str(tmp_path / f"m{k}")
        copy_oracle(work)
        with open(os.path.join(work, "oracle", f), "w") as fh:
            fh.write(src[f].replace(old, new, 1))
        r = run_pins(work, ps)
        # A failed pin (exit 1), not a collection or build error (other codes).
        return name, r.returncode, r.stdout[-1500:]

    with ThreadPoolExecutor(max_workers=6) as ex:
        results = list(ex.map(one, range(len(mutants))))
    survivors = [name for name, rc, _ in results if rc == 0]
    broken = [(name, rc, out) for name, rc, out in results if rc not in (0, 1)]
    assert not broken, broken
    assert not survivors, f"planted mistakes no pin caught: {survivors}"

"""The premise of the FP32 compatibility state of the sweep kernel (CPU only):
S_l - S_r = S(Ql) - S(Qr) for the half-space sign moments S of the
compatibility condition (Sec. 2.1) is replaced, for relative jumps
r = |drho|/rho + |dm|/sqrt(rho p) + (gamma-1)|dE|/p < 2e-3, by the midpoint
rule J_S(Q_m)(Ql - Qr).  With D(t) = S(Q_m + t dQ/2) - S(Q_m - t dQ/2), odd in
t, the rule keeps the linear term of D(1) and drops c3 + c5 + ...; the test
measures that remainder with the oracle's FP64 compatibility state,
c3 ~ (4/3)(D(1) - 2 D(1/2)), and holds it below 3e-9 of |S| (~2e-8
absolute, under the FP32 rounding of Q0) at the threshold, and shows it
growing like r^3."""
import numpy as np

import oracle

GAMMA = 1.4


def S_diff(qm, dq, t):
    # compat(Ql, Qr) = (Ql + Qr)/2 + (S(Ql) - S(Qr))/2
    ql, qr = qm + 0.5 * t * dq, qm - 0.5 * t * dq
    return 2.0 * oracle.compat(ql, qr, GAMMA) - (ql + qr)


def jump_ratio(qm, dq):
    rho = qm[0]
    p = (GAMMA - 1) * (qm[4] - 0.5 * (qm[1:4] ** 2).sum() / rho)
    return (abs(dq[0]) / rho + np.abs(dq[1:4]).sum() / np.sqrt(rho * p)
            + (GAMMA - 1) * abs(dq[4]) / p)


def test_midpoint_rule_remainder_below_threshold():
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-2, 2, 3)
        p = 100 / 1.4 * rng.uniform(0.9, 1.1)  # Ma ~ 0.1-0.3, as in the paper's cases
        qm = np.array([rho, *(rho * u), p / (GAMMA - 1) + 0.5 * rho * (u ** 2).sum()])
        dq = rng.standard_normal(5) * np.array([rho, rho, rho, rho, p])
        dq *= 2e-3 / jump_ratio(qm, dq)  # at the threshold
        s_scale = rho * np.sqrt(2 * (p / rho) / np.pi)  # the size of S
        d1, dh = S_diff(qm, dq, 1.0), S_diff(qm, dq, 0.5)
        c3 = 4.0 / 3.0 * (d1 - 2.0 * dh)
        assert np.abs(c3).max() <= 3e-9 * s_scale, (np.abs(c3).max(), s_scale)
        # and the remainder shrinks like r^3: ten times smaller jump, ~1000x smaller
        d1s, dhs = S_diff(qm, 0.1 * dq, 1.0), S_diff(qm, 0.1 * dq, 0.5)
        c3s = 4.0 / 3.0 * (d1s - 2.0 * dhs)
        big = np.abs(c3).max()
        if big > 1e-12 * s_scale:
            assert np.abs(c3s).max() <= 3e-3 * big + 1e-14 * s_scale

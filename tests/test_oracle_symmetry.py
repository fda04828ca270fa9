"""Symmetries of the whole oracle step (CPU only).

The gas-kinetic step commutes with the symmetries of the box that the
scheme's construction respects: a cyclic relabelling of the axes (the
tangential directions of a face are t1 = d+1, t2 = d+2, so the construction
maps onto itself), a reflection of any one axis (WENO5's right value is the
mirror image of its left value, the half-space moments swap), and, with
linear weights, the exchange of two axes (the tangential reconstruction is
then a tensor product, the same in either order).  Each holds to rounding
on a rectangular box with unequal extents, so a transposed velocity
component, a derivative taken along the wrong axis or width, or a sign
error in one direction fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_08736_gb300 import inputs

N = (6, 7, 8)
L = (1.0, 1.3, 1.7)
DT = 0.02
MODES = [(oracle.RECON_LINEAR, oracle.FLUX_SMOOTH, 0), (oracle.RECON_WENO_JS, oracle.FLUX_FULL, 0),
         (oracle.RECON_WENO_Z, oracle.FLUX_FULL, 0), (oracle.RECON_WENO_Z, oracle.FLUX_FULL, 1)]


def step(Q, n, lens, recon, flux, char):
    s = oracle.Solver(oracle.Config(*n, lx=lens[0], ly=lens[1], lz=lens[2], recon=recon, flux=flux,
                                    tau_num_C=1.0, mu_ref=0.01, char_recon=char))
    s.set_state(np.ascontiguousarray(Q))
    s.step(2, DT)
    return s.state()


def start():
    return oracle.conservative(inputs.random_smooth(N, seed=3, amp=0.2), 1.4)


def cyclic(Q):
    """Relabel (x, y, z) -> (y, z, x): the old z axis becomes x; momentum
    components follow their axes.  Arrays are [var][z][y][x]."""
    return np.transpose(Q, (0, 2, 3, 1))[[0, 3, 1, 2, 4]]


def reflect(Q, axis):
    """Mirror the axis (0 = x, 1 = y, 2 = z) and negate its momentum."""
    R = np.flip(Q, axis=3 - axis).copy()
    R[1 + axis] *= -1
    return R


def swap_xy(Q):
    return np.transpose(Q, (0, 1, 3, 2))[[0, 2, 1, 3, 4]]


@pytest.mark.parametrize("recon,flux,char", MODES)
def test_step_commutes_with_a_cyclic_relabelling_of_the_axes(recon, flux, char):
    Q = start()
    A = step(Q, N, L, recon, flux, char)
    B = step(cyclic(Q), (N[2], N[0], N[1]), (L[2], L[0], L[1]), recon, flux, char)
    assert np.abs(A - Q).max() > 1e-2
    assert np.abs(cyclic(A) - B).max() < 1e-13


@pytest.mark.parametrize("recon,flux,char", MODES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step_commutes_with_a_reflection(recon, flux, char, axis):
    Q = start()
    A = step(Q, N, L, recon, flux, char)
    B = step(reflect(Q, axis), N, L, recon, flux, char)
    assert np.abs(reflect(A, axis) - B).max() < 1e-13


def test_linear_step_commutes_with_an_exchange_of_two_axes():
    Q = start()
    A = step(Q, N, L, oracle.RECON_LINEAR, oracle.FLUX_SMOOTH, 0)
    B = step(swap_xy(Q), (N[1], N[0], N[2]), (L[1], L[0], L[2]), oracle.RECON_LINEAR,
             oracle.FLUX_SMOOTH, 0)
    assert np.abs(swap_xy(A) - B).max() < 1e-13

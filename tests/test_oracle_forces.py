"""Pins of the oracle's analytic gradients to central finite differences.

Each finite difference re-solves the induced dipoles to 1e-13 D, so it
differentiates the full polarization energy U(r, q, d, Theta) including the
response of mu; the analytic gradients are taken at fixed mu. Agreement
therefore also checks that the energy is stationary in mu.
"""
import copy

import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.forces import polarization_gradients
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import WATER_648, make_waters, small_box_settings


def energy(sysm, st):
    op = Operator(sysm, st)
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-13, 500)
    return polarization_energy(mu, e0), op, mu


def shifted(sysm, field, idx, h):
    s = copy.deepcopy(sysm)
    a = getattr(s, field).copy()
    a[idx] += h
    setattr(s, field, a)
    return s


def fd(sysm, st, field, idx, h=1e-5):
    return (energy(shifted(sysm, field, idx, h), st)[0] - energy(shifted(sysm, field, idx, -h), st)[0]) / (2 * h)


CASES = {
    "cluster3": lambda: (make_waters(3, 6.0, 3, periodic=False), Setup.cluster(), [0, 1, 4]),
    "box8": lambda: (make_waters(8, 9.0, 7), Setup(box=9.0, cutoff=small_box_settings(9.0)[0],
                                                   beta=small_box_settings(9.0)[1],
                                                   grid=small_box_settings(9.0)[2]), [0, 5, 13]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_forces_match_finite_differences(name):
    sysm, st, atoms = CASES[name]()
    _, op, mu = energy(sysm, st)
    F, _, _, _ = polarization_gradients(op, mu)
    scale = np.abs(F).max()
    for k in atoms:
        for a in range(3):
            assert -fd(sysm, st, "xyz", (k, a)) == pytest.approx(F[k, a], abs=1e-8 * scale)


@pytest.mark.parametrize("name", sorted(CASES))
def test_moment_gradients_match_finite_differences(name):
    sysm, st, atoms = CASES[name]()
    _, op, mu = energy(sysm, st)
    _, gq, gd, gt = polarization_gradients(op, mu)
    for k in atoms[:2]:
        assert fd(sysm, st, "q", k) == pytest.approx(gq[k], rel=1e-8, abs=1e-10)
        for a in range(3):
            assert fd(sysm, st, "dip", (k, a)) == pytest.approx(gd[k, a], rel=1e-8, abs=1e-10)
        for c in (0, 2, 3, 5):
            assert fd(sysm, st, "quad", (k, c)) == pytest.approx(gt[k, c], rel=1e-7, abs=1e-10)


def test_cluster_forces_sum_to_zero():
    """No external field: the polarization forces of an isolated cluster cancel."""
    sysm = make_waters(5, 8.0, 9, periodic=False)
    _, op, mu = energy(sysm, Setup.cluster())
    F, _, _, _ = polarization_gradients(op, mu)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).max()


def test_forces_648_box_two_atoms():
    w = WATER_648
    sysm = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    _, op, mu = energy(sysm, st)
    F, _, _, _ = polarization_gradients(op, mu)
    scale = np.abs(F).max()
    for k in (3, 400):
        for a in range(3):
            assert -fd(sysm, st, "xyz", (k, a)) == pytest.approx(F[k, a], abs=1e-7 * scale)

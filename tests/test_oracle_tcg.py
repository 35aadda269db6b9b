"""Pins of the oracle's TCG-1 energy and gradients, and of their building blocks.

Expected values come from central finite differences of the oracle's own
energies and fields (re-evaluated from scratch at shifted inputs) and from the
definition of the first conjugate-gradient iterate.
"""
import copy

import numpy as np
import pytest

from oracle import Setup
from oracle.solver import Operator, pcg
from oracle.tcg import bilinear_T_gradient, field_gradients, tcg1, tcg1_gradients
from paper_1906_01211_gb300.synth import make_waters, small_box_settings


def _box8():
    L = 9.0
    rc, beta, K = small_box_settings(L)
    return make_waters(8, L, 7), Setup(box=L, cutoff=rc, beta=beta, grid=K)


CASES = {
    "box8": _box8,
    "cluster4": lambda: (make_waters(4, 6.0, 2, periodic=False), Setup.cluster()),
}


def _shift(s, field, idx, h):
    t = copy.deepcopy(s)
    a = getattr(t, field).copy()
    a[idx] += h
    setattr(t, field, a)
    return t


def _fd(f, s, field, idx, h):
    return (f(_shift(s, field, idx, h)) - f(_shift(s, field, idx, -h))) / (2 * h)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tcg1_iterate_is_the_first_pcg_iterate(name):
    s, st = CASES[name]()
    op = Operator(s, st)
    _, mu1, _ = tcg1(op)
    ref, it, _ = pcg(lambda m: (1 / s.alpha)[:, None] * m - op.apply_T(m), s.alpha, op.permanent_field(), 0.0, 1)
    assert it == 1
    assert np.abs(mu1 - ref).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("name", sorted(CASES))
def test_field_gradients_match_finite_differences(name):
    s, st = CASES[name]()
    c = np.random.default_rng(0).normal(size=(s.n, 3))

    def ce(S):
        return float((c * Operator(S, st).permanent_field()).sum())

    gx, gq, gd, gt = field_gradients(Operator(s, st), c)
    for k in (0, 4):
        for a in range(3):
            assert _fd(ce, s, "xyz", (k, a), 1e-5) == pytest.approx(gx[k, a], rel=1e-6, abs=1e-8 * np.abs(gx).max())
            assert _fd(ce, s, "dip", (k, a), 1e-3) == pytest.approx(gd[k, a], rel=1e-8, abs=1e-10)
        assert _fd(ce, s, "q", k, 1e-3) == pytest.approx(gq[k], rel=1e-8, abs=1e-10)
        for m in (0, 3, 5):
            assert _fd(ce, s, "quad", (k, m), 1e-3) == pytest.approx(gt[k, m], rel=1e-8, abs=1e-10)


@pytest.mark.parametrize("name", sorted(CASES))
def test_bilinear_T_gradient_matches_finite_differences_and_is_symmetric(name):
    s, st = CASES[name]()
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(s.n, 3)), rng.normal(size=(s.n, 3))
    op = Operator(s, st)
    g = bilinear_T_gradient(op, a, b)
    assert np.abs(g - bilinear_T_gradient(op, b, a)).max() < 1e-13 * np.abs(g).max()

    def atb(S):
        return float((a * Operator(S, st).apply_T(b)).sum())

    for k in (1, 7):
        for x in range(3):
            assert _fd(atb, s, "xyz", (k, x), 1e-5) == pytest.approx(g[k, x], rel=1e-6, abs=1e-8 * np.abs(g).max())


@pytest.mark.parametrize("name", sorted(CASES))
def test_tcg1_forces_match_finite_differences(name):
    """U_1 is not stationary in mu_1: the gradient differentiates through gamma,
    r and z, and finite differences of the full TCG-1 energy check all of it."""
    s, st = CASES[name]()

    def u1(S):
        return tcg1(Operator(S, st))[0]

    F, _, _, _ = tcg1_gradients(Operator(s, st))
    scale = np.abs(F).max()
    for k in (0, 5, 10):
        for a in range(3):
            assert -_fd(u1, s, "xyz", (k, a), 1e-5) == pytest.approx(F[k, a], abs=1e-7 * scale)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tcg1_moment_gradients_match_finite_differences(name):
    s, st = CASES[name]()

    def u1(S):
        return tcg1(Operator(S, st))[0]

    _, gq, gd, gt = tcg1_gradients(Operator(s, st))
    h = 1e-4  # U_1 is a ratio of quadratics in the moments: O(h^2) truncation
    for k in (2, 9):
        assert _fd(u1, s, "q", k, h) == pytest.approx(gq[k], rel=1e-6, abs=1e-8)
        for a in range(3):
            assert _fd(u1, s, "dip", (k, a), h) == pytest.approx(gd[k, a], rel=1e-6, abs=1e-8)
        for m in (3, 4, 5):
            assert _fd(u1, s, "quad", (k, m), h) == pytest.approx(gt[k, m], rel=1e-6, abs=1e-8)

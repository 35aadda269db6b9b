"""Pins of the oracle's two-field (direct / polarization scaled) solve.

Expected values come from the one-field oracle (the two fields coincide at
scale 0), from the symmetry of A, from an independent construction of the
field difference out of isolated molecules, and from central finite
differences of the two-field energy.
"""
import copy

import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.solver import Operator, solve
from oracle.two_rhs import permanent_field_scaled, two_rhs_gradients, two_rhs_solve
from paper_1906_01211_gb300.synth import System, make_waters, small_box_settings


def _box8():
    L = 9.0
    rc, beta, K = small_box_settings(L)
    return make_waters(8, L, 7), Setup(box=L, cutoff=rc, beta=beta, grid=K)


CASES = {
    "box8": _box8,
    "cluster4": lambda: (make_waters(4, 6.0, 2, periodic=False), Setup.cluster()),
}


def test_scale_zero_is_the_one_field_problem():
    s, st = _box8()
    op = Operator(s, st)
    U, mu_d, mu_p, e_d, e_p = two_rhs_solve(op, 0.0, 1e-13)
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-13, 500)
    assert np.abs(e_p - e0).max() == 0.0 and np.abs(e_d - e0).max() == 0.0
    assert U == pytest.approx(polarization_energy(mu, e0), rel=1e-12)


@pytest.mark.parametrize("name", sorted(CASES))
def test_energy_is_symmetric_in_the_two_fields(name):
    s, st = CASES[name]()
    _, mu_d, mu_p, e_d, e_p = two_rhs_solve(Operator(s, st), 0.6, 1e-13)
    assert (mu_d * e_p).sum() == pytest.approx((mu_p * e_d).sum(), rel=1e-9)


def test_field_difference_is_the_damped_field_inside_each_molecule():
    """E_p - E_d = s_p x (Thole-damped bare field of a molecule's own sites),
    built here from each water alone as an isolated cluster whose three
    sites are made separate molecules."""
    s, st = _box8()
    op = Operator(s, st)
    sp = 0.35
    diff = permanent_field_scaled(op, sp) - permanent_field_scaled(op, 0.0)
    ref = np.zeros_like(diff)
    for w in range(s.n // 3):
        idx = np.arange(3 * w, 3 * w + 3)
        c = System(xyz=s.xyz[idx], q=s.q[idx], dip=s.dip[idx], quad=s.quad[idx], alpha=s.alpha[idx],
                   thole=s.thole[idx], mol=np.arange(3, dtype=np.int32), box=None)
        ref[idx] = Operator(c, Setup.cluster()).permanent_field()
    assert np.abs(diff - sp * ref).max() < 1e-12 * np.abs(ref).max()


def _shift(s, field, idx, h):
    t = copy.deepcopy(s)
    a = getattr(t, field).copy()
    a[idx] += h
    setattr(t, field, a)
    return t


@pytest.mark.parametrize("name", sorted(CASES))
def test_gradients_match_finite_differences(name):
    s, st = CASES[name]()
    sp = 0.5
    _, mu_d, mu_p, _, _ = two_rhs_solve(Operator(s, st), sp, 1e-13)
    F, gq, gd, gt = two_rhs_gradients(Operator(s, st), sp, mu_d, mu_p)

    def u(S):
        return two_rhs_solve(Operator(S, st), sp, 1e-13)[0]

    def fd(field, idx, h):
        return (u(_shift(s, field, idx, h)) - u(_shift(s, field, idx, -h))) / (2 * h)

    for k in (0, 5):
        for a in range(3):
            assert -fd("xyz", (k, a), 1e-5) == pytest.approx(F[k, a], abs=1e-7 * np.abs(F).max())
            assert fd("dip", (k, a), 1e-3) == pytest.approx(gd[k, a], rel=1e-7, abs=1e-9)
        assert fd("q", k, 1e-3) == pytest.approx(gq[k], rel=1e-7, abs=1e-9)
        for m in (3, 4, 5):
            assert fd("quad", (k, m), 1e-3) == pytest.approx(gt[k, m], rel=1e-7, abs=1e-9)

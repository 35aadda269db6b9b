"""Randomised properties of the oracle on small isolated clusters (hypothesis).

Each example draws a seeded water cluster; the properties hold for every
geometry and every set of moments: invariance of both energies under a rigid
motion that also turns the global-frame moments, no net force on an isolated
cluster, and agreement of the iterative solve with the dense Cholesky solve.
"""
import copy

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import Setup  # noqa: E402
from oracle.energy import polarization_energy  # noqa: E402
from oracle.forces import polarization_gradients  # noqa: E402
from oracle.multipole import multipole_energy  # noqa: E402
from oracle.realspace import quad_matrix  # noqa: E402
from oracle.solver import Operator, dense_solve, rms_debye, solve  # noqa: E402
from paper_1906_01211_gb300.synth import make_waters  # noqa: E402

CLUSTER = Setup.cluster()


def _rotation(u):
    q = np.asarray(u, float)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _turned(s, Q, t):
    """The cluster moved rigidly: x -> Q x + t, d -> Q d, Theta -> Q Theta Q^T."""
    r = copy.deepcopy(s)
    th = np.einsum("ab,pbc,dc->pad", Q, quad_matrix(s.quad), Q)
    r.xyz = s.xyz @ Q.T + t
    r.dip = s.dip @ Q.T
    r.quad = np.stack([th[:, 0, 0], th[:, 1, 1], th[:, 2, 2], th[:, 0, 1], th[:, 0, 2], th[:, 1, 2]], 1)
    return r


def _upol(s):
    op = Operator(s, CLUSTER)
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-12, 500)
    return polarization_energy(mu, e0), op, mu, e0


quat = st.lists(st.floats(-1, 1), min_size=4, max_size=4).filter(lambda v: np.linalg.norm(v) > 0.1)


@settings(max_examples=10, deadline=None)
@given(nw=st.integers(2, 5), seed=st.integers(0, 10_000), q=quat,
       t=st.lists(st.floats(-5, 5), min_size=3, max_size=3))
def test_energies_invariant_under_rigid_motion(nw, seed, q, t):
    s = make_waters(nw, 8.0, seed, periodic=False)
    r = _turned(s, _rotation(q), np.asarray(t))
    assert multipole_energy(r, CLUSTER, False) == pytest.approx(multipole_energy(s, CLUSTER, False), rel=1e-10,
                                                               abs=1e-10)
    assert _upol(r)[0] == pytest.approx(_upol(s)[0], rel=1e-9, abs=1e-10)


@settings(max_examples=10, deadline=None)
@given(nw=st.integers(2, 5), seed=st.integers(0, 10_000))
def test_no_net_force_on_an_isolated_cluster(nw, seed):
    s = make_waters(nw, 8.0, seed, periodic=False)
    _, op, mu, _ = _upol(s)
    F, _, _, _ = polarization_gradients(op, mu)
    assert np.abs(F.sum(0)).max() < 1e-10 * max(np.abs(F).max(), 1e-12)
    _, Fm, _, _, _ = multipole_energy(s, CLUSTER)
    assert np.abs(Fm.sum(0)).max() < 1e-10 * max(np.abs(Fm).max(), 1e-12)


@settings(max_examples=10, deadline=None)
@given(nw=st.integers(1, 4), seed=st.integers(0, 10_000))
def test_pcg_agrees_with_the_dense_solve(nw, seed):
    s = make_waters(nw, 7.0, seed, periodic=False)
    _, op, mu, e0 = _upol(s)
    assert rms_debye(mu - dense_solve(op.apply_A, e0)) < 1e-10

"""The 96,000-atom periodic box (32,000 waters, L = 98.65 A, K = 100) at full
size, float64 and mixed, against the oracle on what it can compute at this
size: the exact pair count, the real-space parts at sampled sites by the
oracle's direct scan, the reciprocal parts in full (oracle PME on the same
grid), and for the solve, the float64 residual at sampled sites (a property
that holds at any size) plus mixed vs float64 on the GPU.

Tolerances as for the smaller boxes: float64 fields 1e-12 relative, mixed
dipoles within 1e-5 D RMS of float64, energy 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.pairs import periodic_pairs
from oracle.pme import PmeGrid, dipole_field_recip, permanent_field_recip, self_field
from oracle.realspace import dipole_field_real_rows, permanent_field_real_rows
from oracle.setup import DEBYE
from paper_1906_01211_gb300.synth import WATER_96000

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def big():
    w = WATER_96000
    sysm = w.system()
    setup = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=5)
    grid = PmeGrid(sysm.xyz, setup.box, setup.grid, setup.order, setup.beta)
    rows = np.random.default_rng(96).choice(sysm.n, 48, replace=False)
    return w, sysm, setup, grid, rows


def solver(w, precision):
    from paper_1906_01211_gb300 import amoebapol as ap
    return ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                     tol_debye=w.tol_debye, precision=precision))


def oracle_T_rows(sysm, setup, grid, v, rows):
    return (dipole_field_real_rows(sysm, setup, v, rows) + dipole_field_recip(sysm, setup, v, grid)[rows]
            + self_field(setup, v)[rows])


def test_96000_pair_count_and_fields(big):
    w, sysm, setup, grid, rows = big
    s = solver(w, "fp64")
    s.set_synthetic(sysm)
    i, _, _ = periodic_pairs(sysm.xyz, w.L, w.cutoff)
    assert s.pair_count() == len(i)
    E0 = s.permanent_field().cpu().numpy()
    ref = (permanent_field_real_rows(sysm, setup, rows) + permanent_field_recip(sysm, setup, grid)[rows]
           + self_field(setup, sysm.dip)[rows])
    assert rel(E0[rows], ref) < 1e-12
    v = np.random.default_rng(7).normal(size=(sysm.n, 3)) * 0.1
    t = s.apply_T(torch.tensor(v)).cpu().numpy()
    assert rel(t[rows], oracle_T_rows(sysm, setup, grid, v, rows)) < 1e-12


def test_96000_solve_residual_and_mixed(big):
    w, sysm, setup, grid, rows = big
    s = solver(w, "fp64")
    s.set_synthetic(sysm)
    E0 = s.permanent_field()
    mu, it, rms = s.solve(E0)
    U = s.energy(mu, E0)
    assert rms < w.tol_debye
    mu_np, E0_np = mu.cpu().numpy(), E0.cpu().numpy()
    # z = alpha (E0 - mu/alpha + T mu) at sampled sites, T mu by the oracle
    Tmu = oracle_T_rows(sysm, setup, grid, mu_np, rows)
    alpha = sysm.alpha[rows, None]
    z = alpha * (E0_np[rows] - mu_np[rows] / alpha + Tmu)
    assert DEBYE * np.sqrt((z * z).sum() / len(rows)) < 3 * w.tol_debye
    m = solver(w, "mixed")
    m.set_synthetic(sysm)
    E0m = m.permanent_field()
    mum, _, rmsm = m.solve(E0m)
    Um = m.energy(mum, E0m)
    d = mum.cpu().numpy() - mu_np
    assert DEBYE * np.sqrt((d * d).sum() / sysm.n) < 1e-5
    assert abs(Um / U - 1) < 1e-6

"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances (float64 path): permanent field and T*mu to 1e-12 relative
(2-norm of the difference over the 2-norm of the oracle vector), induced
dipoles to 1e-8 Debye RMS, energy to 1e-10 relative. Mixed path: dipoles
within 1e-5 Debye RMS of the float64 oracle, energy within 1e-6 relative.
Beside every norm check, a per-atom one (tests/parity_metrics.py): the
largest per-atom field error within the same tolerance relative to the
largest per-atom field, the largest per-atom dipole error within the RMS
tolerance (float64) or 5x it (mixed: its dipoles are converged to 1e-5 D
RMS, so single atoms may sit a few times above that).
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.realspace import dipole_field_real_rows, permanent_field_real_rows
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import (WATER_648, WATER_23556, density_box_edge, make_waters,
                                          small_box_settings)
from tests.parity_metrics import assert_dipoles, assert_fields, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def make_solver(L, rc, beta, K, tol, precision="fp64", max_iter=100):
    from paper_1906_01211_gb300 import amoebapol as ap
    cfg = ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=tol, precision=precision,
                    max_iter=max_iter)
    return ap.Polarization(cfg)


class Case:
    def __init__(self, sysm, L, rc, beta, K, tol):
        self.sys, self.L, self.rc, self.beta, self.K, self.tol = sysm, L, rc, beta, K, tol
        self.setup = Setup(box=L, cutoff=rc, beta=beta, grid=K, order=5)
        self.op = Operator(sysm, self.setup)
        self.E0 = self.op.permanent_field()
        self.mu, self.iters, self.rms = solve(self.op, self.E0, tol)
        self.U = polarization_energy(self.mu, self.E0)


@pytest.fixture(scope="module")
def w648():
    w = WATER_648
    return Case(w.system(), w.L, w.cutoff, w.beta, w.grid, w.tol_debye)


@pytest.fixture(scope="module")
def w23556():
    w = WATER_23556
    return Case(w.system(), w.L, w.cutoff, w.beta, w.grid, w.tol_debye)


def run_gpu(case, precision="fp64"):
    s = make_solver(case.L, case.rc, case.beta, case.K, case.tol, precision)
    s.set_synthetic(case.sys)
    E0 = s.permanent_field()
    mu, it, rms = s.solve(E0)
    U = s.energy(mu, E0)
    torch.cuda.synchronize()
    return s, E0.cpu().numpy(), mu.cpu().numpy(), it, rms, U


def test_pair_count_matches_oracle(w648):
    s = make_solver(w648.L, w648.rc, w648.beta, w648.K, w648.tol)
    s.set_synthetic(w648.sys)
    assert s.pair_count() == w648.op.n_pairs


def test_fp64_permanent_field_648(w648):
    s, E0, _, _, _, _ = run_gpu(w648)
    assert_fields(E0, w648.E0, 1e-12)


def test_fp64_apply_T_648(w648):
    s = make_solver(w648.L, w648.rc, w648.beta, w648.K, w648.tol)
    s.set_synthetic(w648.sys)
    rng = np.random.default_rng(7)
    for _ in range(2):
        mu = rng.normal(size=(w648.sys.n, 3)) * 0.1
        t = s.apply_T(torch.tensor(mu)).cpu().numpy()
        assert_fields(t, w648.op.apply_T(mu), 1e-12)


def test_fp64_solve_and_energy_648(w648):
    s, E0, mu, it, rms, U = run_gpu(w648)
    assert rms < w648.tol
    assert it == w648.iters
    assert_dipoles(mu, w648.mu, 1e-8)
    assert abs(U / w648.U - 1) < 1e-10


def test_fp64_reruns_agree(w648):
    """Reruns differ only in the rounding order of the PME spreading atomics."""
    a = run_gpu(w648)
    b = run_gpu(w648)
    assert rel(a[1], b[1]) < 1e-14 and rel(a[2], b[2]) < 1e-13 and abs(a[5] / b[5] - 1) < 1e-13


def test_mixed_648_within_tolerance_of_fp64_oracle(w648):
    s, E0, mu, it, rms, U = run_gpu(w648, "mixed")
    assert rms < w648.tol
    assert_dipoles(mu, w648.mu, 1e-5, 5.0)
    assert abs(U / w648.U - 1) < 1e-6


def test_fp64_23556_full_vectors(w23556):
    s, E0, mu, it, rms, U = run_gpu(w23556)
    assert s.pair_count() == w23556.op.n_pairs
    assert_fields(E0, w23556.E0, 1e-12)
    rng = np.random.default_rng(3)
    v = rng.normal(size=(w23556.sys.n, 3)) * 0.1
    t = s.apply_T(torch.tensor(v)).cpu().numpy()
    assert_fields(t, w23556.op.apply_T(v), 1e-12)
    assert it == w23556.iters
    assert_dipoles(mu, w23556.mu, 1e-8)
    assert abs(U / w23556.U - 1) < 1e-10


def test_mixed_23556(w23556):
    s, E0, mu, it, rms, U = run_gpu(w23556, "mixed")
    assert_dipoles(mu, w23556.mu, 1e-5, 5.0)
    assert abs(U / w23556.U - 1) < 1e-6


@pytest.mark.parametrize("nw,seed", [(40, 11), (65, 12), (100, 13)])
def test_small_boxes_ragged_sizes(nw, seed):
    """Boxes with one or two cells per axis and atom counts off any tile size."""
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    case = Case(make_waters(nw, L, seed), L, rc, beta, K, 1e-10)
    s, E0, mu, it, rms, U = run_gpu(case)
    assert_fields(E0, case.E0, 1e-12)
    assert_dipoles(mu, case.mu, 1e-8)
    assert abs(U / case.U - 1) < 1e-10


@pytest.mark.parametrize("nw,K", [(300, 16), (300, 18), (300, 20), (300, 30), (1000, 32), (300, 36), (300, 40),
                                  (500, 48), (500, 50), (1000, 60), (300, 72), (300, 80), (300, 96), (300, 100),
                                  (300, 120), (300, 128)])
def test_own_fft_grids(nw, K):
    """Even 2,3,5-smooth grids from 16 to 128 take the own FFT (radix 4, 2,
    5 and 3 stages; clusters of 2 to 8 CTAs per plane): E0 (float64 variant),
    T*mu (double-float variant) and the solve against the oracle."""
    L = density_box_edge(nw)
    rc, beta, _ = small_box_settings(L)
    case = Case(make_waters(nw, L, 40 + K), L, rc, beta, K, 1e-10)
    s, E0, mu, it, rms, U = run_gpu(case)
    assert_fields(E0, case.E0, 1e-12)
    v = np.random.default_rng(K).normal(size=(case.sys.n, 3)) * 0.1
    assert_fields(s.apply_T(torch.tensor(v)).cpu().numpy(), case.op.apply_T(v), 1e-12)
    assert_dipoles(mu, case.mu, 1e-8)


@pytest.mark.parametrize("nw,K", [(300, 48), (300, 72)])
def test_mixed_own_and_library_fft_grids(nw, K):
    """The mixed operator's float32 chain takes the own FFT up to K = 64 and
    cuFFT above; its float64 check takes the own double-float FFT on both."""
    L = density_box_edge(nw)
    rc, beta, _ = small_box_settings(L)
    case = Case(make_waters(nw, L, 60 + K), L, rc, beta, K, 1e-8)
    s, E0, mu, it, rms, U = run_gpu(case, "mixed")
    assert rms < case.tol
    assert_dipoles(mu, case.mu, 1e-5, 5.0)
    assert abs(U / case.U - 1) < 1e-6


def test_isolated_atoms_have_empty_rows():
    """Two waters far apart in a large box: most rows hold only intramolecular pairs,
    the field still includes PME and self terms."""
    from paper_1906_01211_gb300.synth import System
    base = make_waters(2, 6.0, 21, periodic=False)
    xyz = base.xyz.copy()
    xyz[3:] += np.array([15.0, 15.0, 15.0])
    sysm = System(xyz=xyz, q=base.q, dip=base.dip, quad=base.quad, alpha=base.alpha, thole=base.thole,
                  mol=base.mol, box=40.0)
    case = Case(sysm, 40.0, 7.0, 0.5446, 40, 1e-10)
    s, E0, mu, it, rms, U = run_gpu(case)
    assert s.pair_count() == case.op.n_pairs == 6
    # E0 (~1e-4) is what is left after the excluded intramolecular real-space
    # terms and the reciprocal terms (~4e-2) cancel: both are float64 on the
    # GPU, so E0 itself is held to 1e-12 relative.
    assert_fields(E0, case.E0, 1e-12)
    assert_dipoles(mu, case.mu, 1e-8)


def test_sampled_rows_match_direct_scan(w23556):
    """Real-space parts at sampled atoms by the oracle's O(N) direct scan."""
    s = make_solver(w23556.L, w23556.rc, w23556.beta, w23556.K, w23556.tol)
    s.set_synthetic(w23556.sys)
    rng = np.random.default_rng(5)
    rows = rng.choice(w23556.sys.n, 64, replace=False)
    E0 = s.permanent_field().cpu().numpy()
    rec_self = w23556.op.permanent_field_parts()
    real_gpu = E0 - rec_self[1] - rec_self[2]
    ref = permanent_field_real_rows(w23556.sys, w23556.setup, rows)
    assert_fields(real_gpu[rows], ref, 1e-12)
    v = rng.normal(size=(w23556.sys.n, 3)) * 0.1
    t = s.apply_T(torch.tensor(v)).cpu().numpy()
    parts = w23556.op.apply_T_parts(v)
    ref_t = dipole_field_real_rows(w23556.sys, w23556.setup, v, rows)
    assert_fields((t - parts[1] - parts[2])[rows], ref_t, 1e-12)

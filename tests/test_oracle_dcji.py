"""Pins of the oracle's divide-and-conquer Jacobi iterations.

Expected values come from the dense Cholesky solution, from the matrix form
of block Jacobi (mu <- mu + D^-1 (E - A mu), D the block diagonal of A)
written out independently, and from the spectral radius of its iteration
matrix, which fixes whether and how fast the iteration converges.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.dcji import cell_blocks, dcji
from oracle.solver import Operator, dense_matrix, dense_solve, rms_debye
from paper_1906_01211_gb300.synth import density_box_edge, make_waters, small_box_settings


@pytest.fixture(scope="module")
def box64():
    nw = 64
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 5)
    op = Operator(s, Setup(box=L, cutoff=rc, beta=beta, grid=K))
    A = dense_matrix(op.apply_A, s.n)
    return s, op, A, dense_solve(op.apply_A, op.permanent_field())


def _block_diag(A, blocks):
    D = np.zeros_like(A)
    for b in blocks:
        k = np.stack([3 * b, 3 * b + 1, 3 * b + 2], axis=1).reshape(-1)
        D[np.ix_(k, k)] = A[np.ix_(k, k)]
    return D


def test_one_block_is_the_direct_solve(box64):
    s, op, A, ref = box64
    mu, it, _ = dcji(op, cell_blocks(s, 1), 1e-12, 10, A)
    assert it == 1
    assert rms_debye(mu - ref) < 1e-12


@pytest.mark.parametrize("cells", [2, 4])
def test_molecule_blocks_converge_to_the_dense_solution(box64, cells):
    s, op, A, ref = box64
    blocks = cell_blocks(s, cells)
    assert all(len(set(s.mol[b])) * 3 == len(b) for b in blocks)  # whole molecules only
    mu, it, r = dcji(op, blocks, 1e-10, 200, A)
    assert r < 1e-10 and it < 200
    assert rms_debye(mu - ref) < 1e-9


def test_iterates_follow_the_matrix_form(box64):
    s, op, A, _ = box64
    blocks = cell_blocks(s, 2)
    D = _block_diag(A, blocks)
    e = op.permanent_field().reshape(-1)
    mu = np.repeat(s.alpha, 3) * e
    for _ in range(3):
        mu = mu + np.linalg.solve(D, e - A @ mu)
    got, it, _ = dcji(op, blocks, 0.0, 3, A)
    assert it == 3
    assert np.abs(got.reshape(-1) - mu).max() < 1e-12 * np.abs(mu).max()


def test_convergence_rate_is_the_spectral_radius(box64):
    """rho(I - D^-1 A) < 1 for molecule blocks and > 1 for single sites (the
    strong coupling inside a water makes point Jacobi diverge); the observed
    residual reduction per iteration approaches rho."""
    s, op, A, _ = box64
    n3 = A.shape[0]
    rho = {}
    for name, blocks in (("molecules", cell_blocks(s, 4)), ("sites", [np.array([a]) for a in range(s.n)])):
        M = np.eye(n3) - np.linalg.solve(_block_diag(A, blocks), A)
        rho[name] = float(np.abs(np.linalg.eigvals(M)).max())
    assert rho["molecules"] < 1.0 < rho["sites"]
    r = [dcji(op, cell_blocks(s, 4), 0.0, k, A)[2] for k in (15, 20)]
    assert (r[1] / r[0]) ** (1 / 5) == pytest.approx(rho["molecules"], rel=0.05)

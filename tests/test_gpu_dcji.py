"""DC-JI on the GPU (amp_dcji) against the oracle (oracle/dcji.py, pinned in
tests/test_oracle_dcji.py by the dense solve, the matrix form of block
Jacobi and the spectral radius of its iteration matrix).

Both sides build the exact block diagonal of the same operator (the GPU by
one operator application per column), factorise it in float64 and iterate
mu <- mu + D^-1 (E - A mu) from alpha E; the iterates agree to rounding, so
the iteration counts are equal and mu agrees to 1e-10 relative (2-norm and
per atom) at tolerance 1e-10 D, and after a fixed number of iterations.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.dcji import cell_blocks, dcji
from oracle.solver import Operator, dense_matrix
from paper_1906_01211_gb300.synth import density_box_edge, make_waters, small_box_settings
from tests.parity_metrics import assert_fields

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def box64():
    nw = 64
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 5)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    op = Operator(s, st)
    return s, st, op, dense_matrix(op.apply_A, s.n)


def _gpu(s, st, cells, tol, max_iter, cluster=False):
    from paper_1906_01211_gb300 import amoebapol as ap
    cfg = ap.Config(box=0.0, tol_debye=1e-10) if cluster else ap.Config(
        box=st.box, cutoff=st.cutoff, ewald_beta=st.beta, pme_grid=st.grid, tol_debye=1e-10)
    p = ap.Polarization(cfg)
    p.set_synthetic(s)
    E0 = p.permanent_field()
    block_of, nb = ap.cell_blocks(s.xyz, s.mol, 0.0 if cluster else st.box, cells)
    mu, it, rms = p.dcji(E0, block_of, nb, tol, max_iter)
    torch.cuda.synchronize()
    p.close()
    return mu.cpu().numpy(), it, rms


@pytest.mark.parametrize("cells", [1, 2, 4])
def test_dcji_matches_oracle(box64, cells):
    s, st, op, A = box64
    mu_ref, it_ref, r_ref = dcji(op, cell_blocks(s, cells), 1e-10, 200, A)
    mu, it, rms = _gpu(s, st, cells, 1e-10, 200)
    assert it == it_ref
    assert rms < 1e-10 and rms == pytest.approx(r_ref, rel=1e-3, abs=1e-13)
    assert_fields(mu, mu_ref, 1e-10)
    if cells == 1:
        assert it == 1  # one block is the direct solve


def test_fixed_iterations_follow_oracle(box64):
    s, st, op, A = box64
    mu_ref, _, r_ref = dcji(op, cell_blocks(s, 2), 0.0, 3, A)
    mu, it, rms = _gpu(s, st, 2, 0.0, 3)
    assert it == 3
    assert rms == pytest.approx(r_ref, rel=1e-8)
    assert_fields(mu, mu_ref, 1e-10)


def test_dcji_cluster_matches_oracle():
    s = make_waters(40, density_box_edge(40), 7, periodic=False)
    op = Operator(s, Setup.cluster())
    A = dense_matrix(op.apply_A, s.n)
    mu_ref, it_ref, _ = dcji(op, cell_blocks(s, 2), 1e-10, 200, A)
    mu, it, rms = _gpu(s, None, 2, 1e-10, 200, cluster=True)
    assert it == it_ref and rms < 1e-10
    assert_fields(mu, mu_ref, 1e-10)


def test_dcji_rejects_bad_blocks_and_mixed_contexts():
    from paper_1906_01211_gb300 import amoebapol as ap
    nw = 20
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 3)
    for precision in ("fp64", "mixed"):
        p = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, precision=precision))
        p.set_synthetic(s)
        E0 = p.permanent_field()
        block_of, nb = ap.cell_blocks(s.xyz, s.mol, L, 2)
        if precision == "mixed":
            with pytest.raises(ap.AmpError):
                p.dcji(E0, block_of, nb)
        else:
            bad = block_of.copy()
            bad[0] = nb  # outside [0, n_blocks)
            with pytest.raises(ap.AmpError):
                p.dcji(E0, bad, nb)
            with pytest.raises(ap.AmpError):
                p.dcji(E0, block_of, nb + 1)  # an empty block
        p.close()

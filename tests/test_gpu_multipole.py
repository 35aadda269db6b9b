"""Permanent-multipole energy and gradients on the GPU against the oracle.

Element by element on the 648-atom box, on small boxes (a ragged 8-water
box, a charged variant that exercises the neutralising background) and on a
40-water cluster, in both precision modes (float64 results in both); on the 23,556-atom
box the energy and eight sampled atoms against stored oracle values. Also
after a position update that reuses the skin lists, and the argument checks.
Tolerances: energy 1e-10 relative, gradients 1e-10 (2-norm relative).
"""
import copy
import json
import os

import numpy as np
import pytest

from oracle import Setup
from oracle.multipole import multipole_energy
from paper_1906_01211_gb300.synth import WATER_648, WATER_23556, make_waters, small_box_settings

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "multipole_water23556.json")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def solver(L, rc, beta, K, precision="fp64"):
    from paper_1906_01211_gb300 import amoebapol as ap
    return ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=1e-8,
                                     precision=precision))


def gpu_mpole(p):
    U, *g = p.multipole_energy()
    return U, [t.cpu().numpy() for t in g]


def check(U, grads, ref, tol=1e-10):
    assert abs(U / ref[0] - 1) < tol
    for g, r in zip(grads, ref[1:]):
        assert rel(g, r) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_water648_matches_oracle(precision):
    w = WATER_648
    s = w.system()
    ref = multipole_energy(s, Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order))
    p = solver(w.L, w.cutoff, w.beta, w.grid, precision)
    p.set_synthetic(s)
    check(*gpu_mpole(p), ref)


@pytest.mark.parametrize("charged", [False, True])
def test_small_box_matches_oracle(charged):
    L = 9.0
    rc, beta, K = small_box_settings(L)
    s = make_waters(8, L, 7)
    if charged:
        s.q = s.q.copy()
        s.q[3] += 0.25
    ref = multipole_energy(s, Setup(box=L, cutoff=rc, beta=beta, grid=K))
    p = solver(L, rc, beta, K)
    p.set_synthetic(s)
    check(*gpu_mpole(p), ref)


def test_water23556_energy_and_sampled_atoms():
    w = WATER_23556
    with open(GOLDEN) as f:
        gold = json.load(f)
    p = solver(w.L, w.cutoff, w.beta, w.grid)
    p.set_synthetic(w.system())
    U, (F, gq, gd, gt) = gpu_mpole(p)
    assert abs(U / gold["U_kcal_mol"] - 1) < 1e-10
    rows = gold["rows"]
    for got, key in ((F, "F"), (gq, "gq"), (gd, "gd"), (gt, "gquad")):
        assert rel(got[rows], np.array(gold[key])) < 1e-10
    # every atom: the quadrupole gradients carry no diagonal mean
    assert np.abs(gt[:, :3].sum(1)).max() < 1e-11 * np.abs(gt).max()


def test_after_position_update_with_skin():
    w = WATER_648
    s = w.system()
    p = solver(w.L, w.cutoff, w.beta, w.grid)
    p.set_list_skin(1.0)
    p.set_synthetic(s)
    rng = np.random.default_rng(5)
    moved = copy.deepcopy(s)
    moved.xyz = s.xyz + rng.uniform(-0.2, 0.2, size=s.xyz.shape)
    assert p.update_positions(moved.xyz)
    ref = multipole_energy(moved, Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order))
    check(*gpu_mpole(p), ref)


def test_energy_only_and_argument_checks():
    from paper_1906_01211_gb300 import amoebapol as ap
    w = WATER_648
    p = solver(w.L, w.cutoff, w.beta, w.grid)
    with pytest.raises(ap.AmpError):
        p.multipole_energy()  # no system yet
    s = w.system()
    p.set_synthetic(s)
    U_only = p.multipole_energy(gradients=False)
    U, _ = gpu_mpole(p)
    # the float64 grid is spread with atomic adds: equal up to summation order
    assert U_only == pytest.approx(U, rel=1e-13)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_matches_oracle(precision):
    """Isolated cluster: every pair with the bare kernels, nothing else."""
    from paper_1906_01211_gb300 import amoebapol as ap
    s = make_waters(40, 12.0, 4, periodic=False)
    ref = multipole_energy(s, Setup.cluster())
    p = ap.Polarization(ap.Config(box=0.0, tol_debye=1e-8, precision=precision))
    p.set_synthetic(s)
    check(*gpu_mpole(p), ref)


def test_autograd_matches_the_call_and_finite_differences():
    from paper_1906_01211_gb300.torch_api import multipole_energy as mpe
    w = WATER_648
    s = w.system()
    p = solver(w.L, w.cutoff, w.beta, w.grid)
    dev = torch.device("cuda")
    xyz, q, dip, quad = (torch.tensor(a, device=dev, requires_grad=True) for a in (s.xyz, s.q, s.dip, s.quad))
    alpha, thole = torch.tensor(s.alpha, device=dev), torch.tensor(s.thole, device=dev)
    mol = torch.tensor(s.mol, device=dev, dtype=torch.int32)
    U = mpe(p, xyz, q, dip, quad, alpha, thole, mol)
    (2.0 * U).backward()
    p.set_synthetic(s)
    U2, (F, gq, gd, gt) = gpu_mpole(p)
    assert U.item() == pytest.approx(U2, rel=1e-13)
    for got, ref in ((xyz.grad, -2.0 * F), (q.grad, 2.0 * gq), (dip.grad, 2.0 * gd), (quad.grad, 2.0 * gt)):
        assert rel(got.cpu().numpy(), ref) < 1e-13
    h = 1e-5
    with torch.no_grad():
        for k, a in ((5, 0), (300, 2)):
            x = xyz.detach().clone()
            x[k, a] += h
            up = mpe(p, x, q.detach(), dip.detach(), quad.detach(), alpha, thole, mol).item()
            x[k, a] -= 2 * h
            dn = mpe(p, x, q.detach(), dip.detach(), quad.detach(), alpha, thole, mol).item()
            assert -(up - dn) / (2 * h) == pytest.approx(F[k, a], abs=1e-6 * np.abs(F).max())

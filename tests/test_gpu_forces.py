"""Adjoint backward on the GPU: against the oracle gradients and against
central finite differences of the GPU energy (h = 1e-5 Angstrom, 64 random
atoms of the 23,556-atom box, seed 3), and through torch.autograd.

Tolerances: float64 gradients within 1e-10 (2-norm relative) of the oracle;
mixed within 2e-5; finite differences within 1e-6 of the largest force.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.forces import polarization_gradients
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import WATER_648, WATER_23556

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_grads(w, tol):
    s = w.system()
    op = Operator(s, Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order))
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, tol, 500)
    return s, mu, polarization_gradients(op, mu)


def gpu_solver(w, precision="fp64", tol=None):
    from paper_1906_01211_gb300 import amoebapol as ap
    return ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                     tol_debye=tol or w.tol_debye, precision=precision))


@pytest.fixture(scope="module")
def o648():
    return oracle_grads(WATER_648, 1e-10)


@pytest.fixture(scope="module")
def o23556():
    return oracle_grads(WATER_23556, 1e-9)


def gpu_grads_at(w, s, mu, precision="fp64"):
    p = gpu_solver(w, precision)
    p.set_synthetic(s)
    return [t.cpu().numpy() for t in p.forces(torch.tensor(mu))]


@pytest.mark.parametrize("fixture,w", [("o648", WATER_648), ("o23556", WATER_23556)])
def test_fp64_gradients_match_oracle(request, fixture, w):
    s, mu, ref = request.getfixturevalue(fixture)
    got = gpu_grads_at(w, s, mu)
    for g, r in zip(got, ref):
        assert rel(g, r) < 1e-10


def test_mixed_gradients_match_oracle(o23556):
    s, mu, ref = o23556
    got = gpu_grads_at(WATER_23556, s, mu, "mixed")
    for g, r in zip(got, ref):
        assert rel(g, r) < 2e-5


def test_forces_match_finite_differences_64_atoms():
    w = WATER_23556
    s = w.system()
    p = gpu_solver(w, tol=1e-10)
    xyz = torch.tensor(s.xyz, device="cuda")
    args = [torch.tensor(a, device="cuda") for a in (s.q, s.dip, s.quad, s.alpha, s.thole)]
    mol = torch.tensor(s.mol, device="cuda", dtype=torch.int32)

    alpha = args[3]

    def energy(x):
        # variational form C (mu.A mu / 2 - mu.E0): its error is second order in
        # the solver residual, unlike -C mu.E0 / 2, so the quotient is not noise
        p.set_system(x, args[0], args[1], args[2], args[3], args[4], mol)
        E0 = p.permanent_field()
        mu, _, _ = p.solve(E0)
        amu = mu / alpha[:, None] - p.apply_T(mu)
        u = 332.0637133 * (0.5 * (mu * amu).sum() - (mu * E0).sum())
        return float(u), mu

    _, mu = energy(xyz)
    F = p.forces(mu)[0].cpu().numpy()
    scale = np.abs(F).max()
    h = 1e-5
    # The real-space sum is truncated at rc, so the energy jumps when a pair
    # crosses the cutoff: skip atoms with a partner within 3h of rc (the seed-3
    # draw holds one, 7e-6 Angstrom outside).
    rng = np.random.default_rng(3)
    atoms = []
    for k in rng.permutation(s.n):
        d = s.xyz[k] - s.xyz
        d -= w.L * np.rint(d / w.L)
        r = np.sqrt((d * d).sum(1))
        r[k] = 0.0
        if np.abs(r - w.cutoff).min() > 3 * h:
            atoms.append(k)
        if len(atoms) == 64:
            break
    worst = 0.0
    for k in atoms:
        for a in range(3):
            xp = xyz.clone()
            xp[k, a] += h
            xm = xyz.clone()
            xm[k, a] -= h
            fd = -(energy(xp)[0] - energy(xm)[0]) / (2 * h)
            worst = max(worst, abs(fd - F[k, a]))
    assert worst < 1e-6 * scale


def test_autograd_matches_direct_adjoint():
    from paper_1906_01211_gb300.torch_api import polarization_energy
    w = WATER_648
    s = w.system()
    p = gpu_solver(w, tol=1e-10)
    xyz = torch.tensor(s.xyz, device="cuda", requires_grad=True)
    q = torch.tensor(s.q, device="cuda", requires_grad=True)
    dip = torch.tensor(s.dip, device="cuda", requires_grad=True)
    quad = torch.tensor(s.quad, device="cuda", requires_grad=True)
    alpha, thole = torch.tensor(s.alpha, device="cuda"), torch.tensor(s.thole, device="cuda")
    mol = torch.tensor(s.mol, device="cuda", dtype=torch.int32)
    U = polarization_energy(p, xyz, q, dip, quad, alpha, thole, mol)
    gx, gq, gd, gt = torch.autograd.grad(2.0 * U, (xyz, q, dip, quad))
    E0 = p.permanent_field()
    mu, _, _ = p.solve(E0)
    F, rq, rd, rt = p.forces(mu)
    assert torch.allclose(gx, -2.0 * F, rtol=1e-9, atol=1e-12)
    assert torch.allclose(gq, 2.0 * rq, rtol=1e-9, atol=1e-12)
    assert torch.allclose(gd, 2.0 * rd, rtol=1e-9, atol=1e-12)
    assert torch.allclose(gt, 2.0 * rt, rtol=1e-9, atol=1e-12)
    # a charge derivative against the forward energy
    h = 1e-6
    qp, qm = q.detach().clone(), q.detach().clone()
    qp[7] += h
    qm[7] -= h
    up = polarization_energy(p, xyz.detach(), qp, dip.detach(), quad.detach(), alpha, thole, mol)
    um = polarization_energy(p, xyz.detach(), qm, dip.detach(), quad.detach(), alpha, thole, mol)
    assert float((up - um) / (2 * h)) == pytest.approx(float(gq[7]) / 2.0, rel=1e-6)

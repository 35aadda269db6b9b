"""The two-field form (general AMOEBA's direct and polarization fields) on
the GPU against the oracle (oracle/two_rhs.py, pinned in
tests/test_oracle_two_rhs.py by the one-field limit, the symmetry of A, an
isolated-molecule construction and finite differences).

E_p from amp_permanent_field_scaled, both solves through amp_solve_induced,
U = -1/2 C mu_d . E_p through amp_polarization_energy, gradients through
amp_two_rhs_forces. Float64 path, solves to 1e-11 D on both sides: fields
1e-12 relative, energy and gradients 1e-10 (2-norm and per atom).
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.solver import Operator
from oracle.two_rhs import permanent_field_scaled, two_rhs_gradients, two_rhs_solve
from paper_1906_01211_gb300.synth import density_box_edge, make_waters, small_box_settings
from tests.parity_metrics import assert_fields, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nw,seed,s_p", [(64, 3, 0.5), (150, 4, 1.0)])
def test_two_rhs_energy_and_gradients_match_oracle(nw, seed, s_p):
    from paper_1906_01211_gb300 import amoebapol as ap
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, seed)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    op = Operator(s, st)
    U_ref, mud_ref, mup_ref, ed_ref, ep_ref = two_rhs_solve(op, s_p, tol=1e-11)
    F_ref, gq_ref, gd_ref, gt_ref = two_rhs_gradients(op, s_p, mud_ref, mup_ref)
    p = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=1e-11, max_iter=500))
    p.set_synthetic(s)
    Ed = p.permanent_field()
    Ep = p.permanent_field_scaled(s_p)
    mud, _, _ = p.solve(Ed)
    mup, _, _ = p.solve(Ep)
    U = p.energy(mud, Ep)
    F, gq, gd, gt = p.two_rhs_forces(s_p, mud, mup)
    torch.cuda.synchronize()
    p.close()
    assert_fields(Ed.cpu().numpy(), ed_ref, 1e-12)
    assert_fields(Ep.cpu().numpy(), ep_ref, 1e-12)
    assert abs(U / U_ref - 1) < 1e-10
    assert_fields(F.cpu().numpy(), F_ref, 1e-10)
    assert rel(gq.cpu().numpy(), gq_ref) < 1e-10
    assert_fields(gd.cpu().numpy(), gd_ref, 1e-10)
    assert rel(gt.cpu().numpy(), gt_ref) < 1e-10


def test_scale_zero_is_the_direct_field():
    from paper_1906_01211_gb300 import amoebapol as ap
    nw = 40
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 9)
    p = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K))
    p.set_synthetic(s)
    a = p.permanent_field()
    b = p.permanent_field_scaled(0.0)
    torch.cuda.synchronize()
    p.close()
    assert torch.equal(a, b)
    op = Operator(s, Setup(box=L, cutoff=rc, beta=beta, grid=K))
    assert_fields(b.cpu().numpy(), permanent_field_scaled(op, 0.0), 1e-12)

"""TCG-1 on the GPU (amp_tcg1) against the oracle (oracle/tcg.py): the
iterate mu_1, the energy U_1 and its exact gradients (forces and the three
moment gradients), which run through gamma, r and z.

Tolerances: float64 path 1e-10 relative (2-norm and per atom) on every
output, as for the polarization forces; mixed path 2e-5 on the 2-norm and
5x that per atom, the factor the mixed dipoles get (TCG-1 has no float64
refinement: the float32 operator's error reaches the result directly). The
oracle's TCG-1 is pinned by finite differences in tests/test_oracle_tcg.py.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.solver import Operator
from oracle.tcg import tcg1, tcg1_gradients
from paper_1906_01211_gb300.synth import WATER_648, density_box_edge, make_waters, small_box_settings
from tests.parity_metrics import assert_fields, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cases():
    w = WATER_648
    L = density_box_edge(70)
    rc, beta, K = small_box_settings(L)
    return {
        "water-648": (w.system(), Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=5)),
        "box70": (make_waters(70, L, 17), Setup(box=L, cutoff=rc, beta=beta, grid=K, order=5)),
    }


def gpu_tcg(sysm, st, precision):
    from paper_1906_01211_gb300 import amoebapol as ap
    p = ap.Polarization(ap.Config(box=st.box, cutoff=st.cutoff, ewald_beta=st.beta, pme_grid=st.grid,
                                  tol_debye=1e-8, precision=precision))
    p.set_synthetic(sysm)
    E0 = p.permanent_field()
    out = p.tcg1(E0)
    torch.cuda.synchronize()
    mu, U, F, gq, gd, gt = out
    res = (mu.cpu().numpy(), U, F.cpu().numpy(), gq.cpu().numpy(), gd.cpu().numpy(), gt.cpu().numpy())
    p.close()
    return res


@pytest.mark.parametrize("name", ["water-648", "box70"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_tcg1_energy_and_gradients_match_oracle(name, precision, tol):
    sysm, st = cases()[name]
    op = Operator(sysm, st)
    U_ref, mu_ref, _ = tcg1(op)
    F_ref, gq_ref, gd_ref, gt_ref = tcg1_gradients(op)
    mu, U, F, gq, gd, gt = gpu_tcg(sysm, st, precision)
    f = 1.0 if precision == "fp64" else 5.0
    assert abs(U / U_ref - 1) < tol
    assert_fields(mu, mu_ref, tol, f)
    assert_fields(F, F_ref, tol, f)
    assert rel(gq, gq_ref) < tol
    assert_fields(gd, gd_ref, tol, f)
    assert rel(gt, gt_ref) < tol


def test_tcg1_cluster_energy():
    from paper_1906_01211_gb300 import amoebapol as ap
    s = make_waters(60, density_box_edge(60), 5, periodic=False)
    op = Operator(s, Setup.cluster())
    U_ref, mu_ref, _ = tcg1(op)
    p = ap.Polarization(ap.Config(box=0.0, tol_debye=1e-8))
    p.set_synthetic(s)
    E0 = p.permanent_field()
    mu, U, *_ = p.tcg1(E0, gradients=False)
    assert abs(U / U_ref - 1) < 1e-10
    assert_fields(mu.cpu().numpy(), mu_ref, 1e-10)
    with pytest.raises(ap.AmpError):
        p.tcg1(E0)  # gradients need a periodic context
    p.close()


def test_tcg1_differs_from_converged_energy():
    """TCG-1 is one step: its energy is above (less negative than) the converged one."""
    sysm, st = cases()["water-648"]
    from paper_1906_01211_gb300 import amoebapol as ap
    p = ap.Polarization(ap.Config(box=st.box, cutoff=st.cutoff, ewald_beta=st.beta, pme_grid=st.grid,
                                  tol_debye=1e-8))
    p.set_synthetic(sysm)
    E0 = p.permanent_field()
    _, U1, *_ = p.tcg1(E0, gradients=False)
    mu, _, _ = p.solve(E0)
    U = p.energy(mu, E0)
    p.close()
    assert U < U1 < 0.0

"""Isolated clusters and the continuous-batching server on the GPU.

Clusters (box = 0: every pair, no Ewald) against the oracle: float64 to 1e-12
relative on E0 and T*mu and 1e-8 D on the dipoles; mixed to 1e-5 D and 1e-6
relative energy. Serving: every request's result is the same alone and in a
mix of concurrent requests, within 1e-5 D RMS and 1e-6 relative energy.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.setup import DEBYE
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import density_box_edge, make_waters

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rms_d(a, b):
    d = np.asarray(a) - np.asarray(b)
    return float(DEBYE * np.sqrt((d * d).sum() / d.shape[0]))


@pytest.mark.parametrize("nw,seed", [(40, 1), (301, 2)])
def test_cluster_fp64_matches_oracle(nw, seed):
    from paper_1906_01211_gb300 import amoebapol as ap
    s = make_waters(nw, density_box_edge(nw), seed, periodic=False)
    op = Operator(s, Setup.cluster())
    e_ref = op.permanent_field()
    mu_ref, it_ref, _ = solve(op, e_ref, 1e-9)
    p = ap.Polarization(ap.Config(box=0.0, tol_debye=1e-9))
    p.set_synthetic(s)
    E0 = p.permanent_field().cpu().numpy()
    assert rel(E0, e_ref) < 1e-12
    v = np.random.default_rng(0).normal(size=(s.n, 3)) * 0.1
    assert rel(p.apply_T(torch.tensor(v)).cpu().numpy(), op.apply_T(v)) < 1e-12
    mu, it, rms = p.solve(torch.tensor(e_ref))
    assert it == it_ref
    assert rms_d(mu.cpu().numpy(), mu_ref) < 1e-8
    assert p.pair_count() == s.n * (s.n - 1) // 2


def test_cluster_mixed_matches_oracle():
    """Same 1e-5 D tolerance on both sides: the energy -C mu.E0/2 carries a
    first-order error of that size, so a tighter reference would measure the
    tolerance, not the precision."""
    from paper_1906_01211_gb300 import amoebapol as ap
    s = make_waters(500, density_box_edge(500), 3, periodic=False)
    op = Operator(s, Setup.cluster())
    e_ref = op.permanent_field()
    mu_ref, _, _ = solve(op, e_ref, 1e-5)
    u_ref = polarization_energy(mu_ref, e_ref)
    p = ap.Polarization(ap.Config(box=0.0, tol_debye=1e-5, precision="mixed"))
    p.set_synthetic(s)
    E0 = p.permanent_field()
    mu, it, rms = p.solve(E0)
    assert rms_d(mu.cpu().numpy(), mu_ref) < 1e-5
    assert abs(p.energy(mu, E0) / u_ref - 1) < 1e-6


def test_reconfigure_reuses_a_context_across_box_sizes():
    from paper_1906_01211_gb300 import amoebapol as ap
    from paper_1906_01211_gb300.synth import small_box_settings
    a, b = make_waters(100, density_box_edge(100), 5), make_waters(110, density_box_edge(110), 6)
    ra, rb = small_box_settings(a.box), small_box_settings(b.box)
    assert ra[2] == rb[2]  # same grid size, different box
    cfg = lambda s, r: ap.Config(box=s.box, cutoff=r[0], ewald_beta=r[1], pme_grid=r[2], tol_debye=1e-9)
    p = ap.Polarization(cfg(a, ra))
    p.reconfigure(cfg(b, rb))
    p.set_synthetic(b)
    e = p.permanent_field().cpu().numpy()
    op = Operator(b, Setup(box=b.box, cutoff=rb[0], beta=rb[1], grid=rb[2]))
    assert rel(e, op.permanent_field()) < 1e-12


def test_served_results_same_alone_and_in_mix():
    from paper_1906_01211_gb300.serve import Server, request_stream
    mix = request_stream(24, seed=11, max_waters=1200)
    probes = [make_waters(300, density_box_edge(300), 21), make_waters(250, density_box_edge(250), 22,
                                                                       periodic=False)]
    alone = []
    srv = Server(n_slots=1, precision="mixed", tol_debye=1e-5)
    for s in probes:
        r = srv.result(srv.submit(s), timeout=120)
        assert r.ok, r.error
        alone.append(r)
    srv.close()
    srv = Server(n_slots=4, precision="mixed", tol_debye=1e-5)
    ids = [srv.submit(s) for s in mix[:12]]
    pid = [srv.submit(s) for s in probes]
    ids += [srv.submit(s) for s in mix[12:]]
    res = {i: srv.result(i, timeout=300) for i in ids + pid}
    srv.close()
    assert all(r.ok for r in res.values()), [r.error for r in res.values() if not r.ok]
    assert max(r.slot for r in res.values()) > 0  # several slots took work
    for a, i in zip(alone, pid):
        b = res[i]
        assert rms_d(a.mu, b.mu) < 1e-5
        assert abs(a.energy / b.energy - 1) < 1e-6


def test_warm_start_from_resident_dipoles():
    from paper_1906_01211_gb300.serve import Server
    s = make_waters(400, density_box_edge(400), 31)
    srv = Server(n_slots=2, precision="mixed", tol_debye=1e-5)
    r1 = srv.result(srv.submit(s, key="w400"), timeout=120)
    r2 = srv.result(srv.submit(s, key="w400"), timeout=120)
    srv.close()
    assert r1.ok and r2.ok and r2.warm_start and not r1.warm_start
    assert r2.iters < r1.iters
    assert rms_d(r1.mu, r2.mu) < 1e-5

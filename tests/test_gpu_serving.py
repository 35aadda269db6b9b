"""Isolated clusters and the continuous-batching server on the GPU.

Clusters (box = 0: every pair, no Ewald) against the oracle: float64 to 1e-12
relative on E0 and T*mu and 1e-8 D on the dipoles; mixed to 1e-5 D and 1e-6
relative energy. Serving: every request's result is the same alone and in a
mix of concurrent requests, within 1e-5 D RMS and 1e-6 relative energy.
Each norm check has a per-atom check beside it (tests/parity_metrics.py;
mixed dipoles: 5x the RMS tolerance per atom).
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import density_box_edge, make_waters
from tests.parity_metrics import assert_dipoles, assert_fields

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    assert_fields(E0, e_ref, 1e-12)
    v = np.random.default_rng(0).normal(size=(s.n, 3)) * 0.1
    assert_fields(p.apply_T(torch.tensor(v)).cpu().numpy(), op.apply_T(v), 1e-12)
    mu, it, rms = p.solve(torch.tensor(e_ref))
    assert it == it_ref
    assert_dipoles(mu.cpu().numpy(), mu_ref, 1e-8)
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
    assert_dipoles(mu.cpu().numpy(), mu_ref, 1e-5, 5.0)
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
    assert_fields(e, op.permanent_field(), 1e-12)


def test_batched_clusters_match_oracle():
    """Small clusters go through the batched engine (persistent kernels over
    the device work queue); each result against the oracle run to the same
    tolerance."""
    from paper_1906_01211_gb300.serve import Server
    systems = [make_waters(nw, density_box_edge(nw), 60 + nw, periodic=False) for nw in (21, 64, 150, 333)]
    with Server(n_workers=1, precision="mixed", tol_debye=1e-5) as srv:
        ids = [srv.submit(s) for s in systems]
        res = [srv.result(i, timeout=120) for i in ids]
        st = srv.stats()
    assert st["batch_launches"] > 0
    for s, r in zip(systems, res):
        assert r.ok, r.error
        assert r.path == "batched"
        op = Operator(s, Setup.cluster())
        e_ref = op.permanent_field()
        mu_ref, it_ref, _ = solve(op, e_ref, 1e-5)
        assert_dipoles(r.mu, mu_ref, 1e-5, 5.0)
        assert abs(r.energy / polarization_energy(mu_ref, e_ref) - 1) < 1e-6
        assert r.rms_debye < 1e-5


def test_served_results_same_alone_and_in_mix():
    """Each probe alone on a fresh server, then among 24 requests of the
    stream's mix (clusters in the batched engine, boxes and large clusters on
    the workers): the same result. On the batched engine it is bit for bit
    the same (every request's sums are taken in a fixed order)."""
    from paper_1906_01211_gb300.serve import Server, request_stream
    mix = request_stream(24, seed=11, max_waters=1200)
    probes = [make_waters(300, density_box_edge(300), 21), make_waters(250, density_box_edge(250), 22,
                                                                       periodic=False)]
    alone = []
    for s in probes:
        with Server(n_workers=1, precision="mixed", tol_debye=1e-5) as srv:
            r = srv.result(srv.submit(s), timeout=120)
        assert r.ok, r.error
        alone.append(r)
    with Server(n_workers=4, precision="mixed", tol_debye=1e-5) as srv:
        ids = [srv.submit(s) for s in mix[:12]]
        pid = [srv.submit(s) for s in probes]
        ids += [srv.submit(s) for s in mix[12:]]
        res = {i: srv.result(i, timeout=300) for i in ids + pid}
    assert all(r.ok for r in res.values()), [r.error for r in res.values() if not r.ok]
    assert {r.path for r in res.values()} == {"batched", "worker"}
    for a, i in zip(alone, pid):
        b = res[i]
        assert a.path == b.path
        assert_dipoles(a.mu, b.mu, 1e-5, 5.0)
        assert abs(a.energy / b.energy - 1) < 1e-6
        if a.path == "batched":
            assert np.array_equal(a.mu, b.mu) and a.energy == b.energy and a.iters == b.iters


def test_warm_start_from_resident_dipoles():
    from paper_1906_01211_gb300.serve import Server
    s = make_waters(400, density_box_edge(400), 31)
    with Server(n_workers=2, precision="mixed", tol_debye=1e-5) as srv:
        r1 = srv.result(srv.submit(s, key="w400"), timeout=120)
        r2 = srv.result(srv.submit(s, key="w400"), timeout=120)
    assert r1.ok and r2.ok and r2.warm_start and not r1.warm_start
    assert r2.iters < r1.iters
    assert_dipoles(r1.mu, r2.mu, 1e-5, 5.0)


def test_bad_and_oversize_requests_fail_alone():
    """Failures made on the host: a site with alpha = 0 and a request larger
    than the whole memory budget each fail alone; the others complete."""
    from paper_1906_01211_gb300.serve import Server
    bad = make_waters(30, density_box_edge(30), 41)
    bad.alpha = bad.alpha.copy()
    bad.alpha[4] = 0.0
    big = make_waters(4000, density_box_edge(4000), 42)
    good = [make_waters(60, density_box_edge(60), 43), make_waters(60, density_box_edge(60), 44, periodic=False)]
    with Server(n_workers=2, precision="mixed", tol_debye=1e-5, mem_budget_bytes=150 << 20,
                batch_arena_atoms=1 << 14, batch_max_requests=64) as srv:
        ids = [srv.submit(good[0]), srv.submit(bad), srv.submit(big), srv.submit(good[1])]
        res = [srv.result(i, timeout=120) for i in ids]
        st = srv.stats()
    assert res[0].ok and res[3].ok
    assert not res[1].ok and "alpha" in res[1].error
    assert not res[2].ok and "budget" in res[2].error
    assert st["failed"] == 2 and st["done"] == 2

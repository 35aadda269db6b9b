"""Local-frame multipoles on the GPU (amp_frames_to_global, amp_frame_forces)
against the oracle (oracle/frames.py, pinned by rigid-motion invariance,
torque balance and finite differences in tests/test_oracle_frames.py).

* the global moments of AMOEBA-water frames (bisector O, Z-then-X H) on a
  700-site box, and sites the call must leave alone (kind -1, axis atoms out
  of range): float64, 1e-14 relative;
* the frame forces from given moment gradients: 1e-12 relative;
* end to end, the total polarization forces of a box with local-frame
  moments (moment gradients from amp_forces, then the frame terms) against
  the oracle's forces plus its frame terms: 1e-10 relative.
"""
import numpy as np
import pytest

from oracle import Setup
from oracle.forces import polarization_gradients
from oracle.frames import frame_forces, global_moments
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import density_box_edge, make_waters, small_box_settings, water_frames
from tests.parity_metrics import assert_fields

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype=None):
    t = torch.tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def test_global_moments_match_oracle():
    from paper_1906_01211_gb300 import amoebapol as ap
    nw = 240
    s = make_waters(nw, density_box_edge(nw), 3)
    kind, za, xa = water_frames(nw)
    kind = kind.copy()
    za = za.copy()
    kind[5] = -1   # global as given
    za[7] = 10**6  # axis atom out of range: left as given
    d_ref, q_ref = global_moments(s.xyz, s.dip, s.quad, np.where(np.arange(s.n) == 7, -1, kind), za, xa)
    dip, quad = ap.frames_to_global(dev(s.xyz), dev(s.dip), dev(s.quad), dev(kind, torch.int32),
                                    dev(za, torch.int32), dev(xa, torch.int32))
    torch.cuda.synchronize()
    assert_fields(dip.cpu().numpy(), d_ref, 1e-14)
    assert np.abs(quad.cpu().numpy() - q_ref).max() < 1e-14 * np.abs(q_ref).max()
    assert np.array_equal(dip.cpu().numpy()[[5, 7]], s.dip[[5, 7]])


def test_frame_forces_match_oracle():
    from paper_1906_01211_gb300 import amoebapol as ap
    nw = 240
    s = make_waters(nw, density_box_edge(nw), 4)
    kind, za, xa = water_frames(nw)
    rng = np.random.default_rng(9)
    gd, gt = rng.normal(size=(s.n, 3)), rng.normal(size=(s.n, 6))
    ref = frame_forces(s.xyz, s.dip, s.quad, kind, za, xa, gd, gt)
    F = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    ap.add_frame_forces(F, dev(s.xyz), dev(s.dip), dev(s.quad), dev(kind, torch.int32), dev(za, torch.int32),
                        dev(xa, torch.int32), dev(gd), dev(gt))
    torch.cuda.synchronize()
    assert_fields(F.cpu().numpy(), ref, 1e-12)


def test_polarization_forces_with_frames_match_oracle():
    from paper_1906_01211_gb300 import amoebapol as ap
    nw = 100
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 8)
    kind, za, xa = water_frames(nw)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    # oracle: global moments from the local ones, solve, fixed-frame gradients + frame terms
    g = make_waters(nw, L, 8)
    g.dip, g.quad = global_moments(s.xyz, s.dip, s.quad, kind, za, xa)
    op = Operator(g, st)
    e0 = op.permanent_field()
    mu_ref, _, _ = solve(op, e0, 1e-12, 500)
    Fd, _, gd, gt = polarization_gradients(op, mu_ref)
    F_ref = Fd + frame_forces(s.xyz, s.dip, s.quad, kind, za, xa, gd, gt)
    # GPU: the same chain through the C ABI
    p = ap.Polarization(ap.Config(box=L, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=1e-12, max_iter=500))
    x, dl, ql = dev(s.xyz), dev(s.dip), dev(s.quad)
    kk, zz, xx = dev(kind, torch.int32), dev(za, torch.int32), dev(xa, torch.int32)
    dip, quad = ap.frames_to_global(x, dl, ql, kk, zz, xx)
    p.set_system(x, s.q, dip, quad, s.alpha, s.thole, s.mol)
    E0 = p.permanent_field()
    mu, _, _ = p.solve(E0)
    F, gq, gdg, gtg = p.forces(mu)
    ap.add_frame_forces(F, x, dl, ql, kk, zz, xx, gdg, gtg)
    torch.cuda.synchronize()
    p.close()
    assert_fields(F.cpu().numpy(), F_ref, 1e-10)

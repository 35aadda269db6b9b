"""Pins of the oracle's local-frame multipoles and frame forces.

Expected values come from properties the frames must have (orthonormal,
right-handed, turning with the molecule), from the invariance of the energy
under rigid motions of an isolated cluster, and from central finite
differences of energies whose moments are rebuilt from the frames at every
shifted geometry.
"""
import copy

import numpy as np
import pytest

from oracle import Setup
from oracle.energy import polarization_energy
from oracle.forces import polarization_gradients
from oracle.frames import frame_forces, frame_jacobian, frames, global_moments
from oracle.multipole import multipole_energy
from oracle.solver import Operator, solve
from paper_1906_01211_gb300.synth import make_waters, small_box_settings, water_frames


def local_system(nw, L, seed, periodic):
    s = make_waters(nw, L, seed, periodic=periodic)
    kind, za, xa = water_frames(nw)
    return s, kind, za, xa


def with_frames(s, kind, za, xa, xyz=None):
    """Copy of s at positions xyz with the global moments of its local ones."""
    t = copy.deepcopy(s)
    if xyz is not None:
        t.xyz = xyz
    t.dip, t.quad = global_moments(t.xyz, s.dip, s.quad, kind, za, xa)
    return t


def rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_frames_are_orthonormal_right_handed_and_follow_the_molecule():
    s, kind, za, xa = local_system(5, 9.0, 3, False)
    R = frames(s.xyz, kind, za, xa)
    assert np.abs(np.einsum("pba,pbc->pac", R, R) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-14
    Q = rotation(1)
    R2 = frames(s.xyz @ Q.T + np.array([0.3, -1.2, 2.0]), kind, za, xa)
    assert np.abs(R2 - np.einsum("ab,pbc->pac", Q, R)).max() < 1e-13
    # bisector: e_z bisects the two O-H directions; Z-then-X: e_z points at the oxygen
    o, h1, h2 = s.xyz[0], s.xyz[1], s.xyz[2]
    u1, u2 = (h1 - o) / np.linalg.norm(h1 - o), (h2 - o) / np.linalg.norm(h2 - o)
    assert np.abs(R[0][:, 2] - (u1 + u2) / np.linalg.norm(u1 + u2)).max() < 1e-14
    assert np.abs(R[1][:, 2] - (o - h1) / np.linalg.norm(o - h1)).max() < 1e-14


def test_frame_jacobian_matches_finite_differences():
    s, kind, za, xa = local_system(3, 9.0, 4, False)
    jac = frame_jacobian(s.xyz, kind, za, xa)
    h = 1e-6
    for i in (0, 1, 5):
        for k, J in jac[i]:
            for c in range(3):
                xp, xm = s.xyz.copy(), s.xyz.copy()
                xp[k, c] += h
                xm[k, c] -= h
                fd = (frames(xp, kind, za, xa)[i] - frames(xm, kind, za, xa)[i]) / (2 * h)
                assert np.abs(fd - J[c]).max() < 1e-7


def test_energies_invariant_under_rigid_motion_of_a_cluster():
    s, kind, za, xa = local_system(4, 8.0, 5, False)
    st = Setup.cluster()
    Q, t = rotation(2), np.array([1.0, -2.0, 0.5])
    a, b = with_frames(s, kind, za, xa), with_frames(s, kind, za, xa, s.xyz @ Q.T + t)
    assert multipole_energy(b, st, False) == pytest.approx(multipole_energy(a, st, False), rel=1e-12)

    def upol(x):
        op = Operator(x, st)
        e0 = op.permanent_field()
        mu, _, _ = solve(op, e0, 1e-12, 500)
        return polarization_energy(mu, e0)

    assert upol(b) == pytest.approx(upol(a), rel=1e-10)


def _mpole_total(s, kind, za, xa, st):
    g = with_frames(s, kind, za, xa)
    U, F, gq, gd, gt = multipole_energy(g, st)
    return U, F + frame_forces(s.xyz, s.dip, s.quad, kind, za, xa, gd, gt)


def test_cluster_forces_and_torques_vanish_with_frame_terms():
    """An isolated cluster feels no net force or torque. With local-frame
    moments the torque balance holds only once the frame terms are added."""
    s, kind, za, xa = local_system(5, 9.0, 6, False)
    st = Setup.cluster()
    g = with_frames(s, kind, za, xa)
    _, Fd, _, gd, gt = multipole_energy(g, st)
    F = Fd + frame_forces(s.xyz, s.dip, s.quad, kind, za, xa, gd, gt)
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-12 * scale
    assert np.abs(np.cross(s.xyz, F).sum(0)).max() < 1e-11 * scale * np.abs(s.xyz).max()
    assert np.abs(np.cross(s.xyz, Fd).sum(0)).max() > 1e-3 * scale


@pytest.mark.parametrize("periodic", [False, True])
def test_multipole_forces_with_frames_match_finite_differences(periodic):
    L = 9.0
    s, kind, za, xa = local_system(8 if periodic else 4, L, 7, periodic)
    if periodic:
        rc, beta, K = small_box_settings(L)
        st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    else:
        st = Setup.cluster()
    _, F = _mpole_total(s, kind, za, xa, st)
    h = 1e-5
    for k in (0, 1, 5):
        for c in range(3):
            xp, xm = s.xyz.copy(), s.xyz.copy()
            xp[k, c] += h
            xm[k, c] -= h
            up = multipole_energy(with_frames(s, kind, za, xa, xp), st, False)
            dn = multipole_energy(with_frames(s, kind, za, xa, xm), st, False)
            assert -(up - dn) / (2 * h) == pytest.approx(F[k, c], abs=1e-7 * np.abs(F).max())


def test_polarization_forces_with_frames_match_finite_differences():
    L = 9.0
    s, kind, za, xa = local_system(8, L, 8, True)
    rc, beta, K = small_box_settings(L)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)

    def upol(x):
        op = Operator(x, st)
        e0 = op.permanent_field()
        mu, _, _ = solve(op, e0, 1e-13, 500)
        return polarization_energy(mu, e0), op, mu

    g = with_frames(s, kind, za, xa)
    _, op, mu = upol(g)
    Fd, _, gd, gt = polarization_gradients(op, mu)
    F = Fd + frame_forces(s.xyz, s.dip, s.quad, kind, za, xa, gd, gt)
    h = 1e-5
    for k in (0, 2, 9):
        for c in range(3):
            xp, xm = s.xyz.copy(), s.xyz.copy()
            xp[k, c] += h
            xm[k, c] -= h
            up = upol(with_frames(s, kind, za, xa, xp))[0]
            dn = upol(with_frames(s, kind, za, xa, xm))[0]
            assert -(up - dn) / (2 * h) == pytest.approx(F[k, c], abs=1e-7 * np.abs(F).max())

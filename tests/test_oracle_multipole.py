"""Pins of the oracle's permanent-multipole energy and gradients.

Every expected value comes from a closed form of classical electrostatics, the
exact Ewald definition, finite differences or an identity the energy must
obey; none is the oracle compared with itself.
"""
import copy
import itertools

import numpy as np
import pytest

from oracle import Setup
from oracle.ewald import screened_B
from oracle.ewald_exact import multipole_energy_exact
from oracle.multipole import _pairings, derivative_tensor, multipole_energy, multipole_rows
from oracle.setup import COULOMB
from paper_1906_01211_gb300.synth import (WATER_648, System, density_box_edge, make_waters,
                                          small_box_settings)


def pair_cluster(ri, rj, qi=0.0, qj=0.0, di=(0, 0, 0), dj=(0, 0, 0), ti=(0,) * 6, tj=(0,) * 6, same=False):
    return System(xyz=np.array([ri, rj], float), q=np.array([qi, qj], float),
                  dip=np.array([di, dj], float), quad=np.array([ti, tj], float),
                  alpha=np.array([0.837, 0.496]), thole=np.array([0.39, 0.39]),
                  mol=np.array([0, 0 if same else 1], np.int32), box=None)


def energy(s, st=None):
    return multipole_energy(s, st or Setup.cluster(), with_gradients=False)


# ---------------------------------------------------------------- derivative tensors

def test_pairings_are_the_involution_numbers():
    """Ways to choose disjoint index pairs among n positions: 1, 1, 2, 4, 10, 26."""
    assert [len(_pairings(n)) for n in range(6)] == [1, 1, 2, 4, 10, 26]


@pytest.mark.parametrize("beta", [0.0, 0.5446])
def test_derivative_tensor_is_the_gradient_of_the_previous_one(beta):
    rng = np.random.default_rng(1)
    r = rng.normal(size=(5, 3)) * 1.5 + np.array([2.0, 0.0, 0.0])
    h = 1e-5

    def T(rr, n):
        d = np.sqrt((rr * rr).sum(1))
        return derivative_tensor(rr, screened_B(d, beta, n), n)

    for n in range(5):
        t1 = T(r, n + 1)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (T(r + e, n) - T(r - e, n)) / (2 * h)
            assert np.allclose(t1[(Ellipsis, c)], fd, rtol=1e-6, atol=1e-8 * np.abs(t1).max())


def test_bare_derivative_tensors_are_traceless():
    """1/r is harmonic away from the origin: every trace of grad^n (1/r) vanishes."""
    r = np.array([[0.7, -1.2, 2.1], [1.9, 0.3, -0.4]])
    d = np.sqrt((r * r).sum(1))
    for n in range(2, 6):
        t = derivative_tensor(r, screened_B(d, 0.0, n), n)
        tr = np.einsum("pii...->p...", t)
        assert np.abs(tr).max() < 1e-12 * np.abs(t).max()


# ---------------------------------------------------------------- closed forms (clusters)

def test_charge_charge_is_coulomb():
    s = pair_cluster([0, 0, 0], [0.3, -1.1, 2.0], qi=0.7, qj=-0.4)
    assert energy(s) == pytest.approx(COULOMB * 0.7 * -0.4 / np.linalg.norm([0.3, -1.1, 2.0]), rel=1e-14)


def test_charge_dipole_and_dipole_dipole():
    ri, rj = np.array([0.4, 1.0, -0.3]), np.array([-1.2, 0.5, 1.7])
    r = ri - rj
    rn = np.linalg.norm(r)
    di, dj = np.array([0.05, -0.02, 0.03]), np.array([-0.04, 0.01, 0.06])
    # charge i in the potential of dipole j: q_i (d_j . r) / r^3
    s = pair_cluster(ri, rj, qi=0.5, dj=dj)
    assert energy(s) == pytest.approx(COULOMB * 0.5 * dj @ r / rn ** 3, rel=1e-13)
    # dipole i in the potential of charge j: d_i . grad(q_j / |r|) = -q_j (d_i . r) / r^3
    s = pair_cluster(ri, rj, qj=-0.3, di=di)
    assert energy(s) == pytest.approx(COULOMB * 0.3 * di @ r / rn ** 3, rel=1e-13)
    s = pair_cluster(ri, rj, di=di, dj=dj)
    expect = COULOMB * (di @ dj / rn ** 3 - 3 * (di @ r) * (dj @ r) / rn ** 5)
    assert energy(s) == pytest.approx(expect, rel=1e-13)


def test_charge_quadrupole_buckingham():
    """A Buckingham quadrupole's potential is (r . Theta . r) / r^5."""
    t = np.array([0.2, -0.5, 0.3, 0.1, -0.05, 0.15])
    th = np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])
    ri, rj = np.array([1.3, -0.2, 0.8]), np.array([0.0, 0.4, -0.9])
    r = ri - rj
    s = pair_cluster(ri, rj, qi=0.6, tj=t)
    assert energy(s) == pytest.approx(COULOMB * 0.6 * (r @ th @ r) / np.linalg.norm(r) ** 5, rel=1e-13)


def test_axial_quadrupoles_on_a_common_axis():
    """Two axial quadrupoles on their common axis: U = 6 Theta_a Theta_b / R^5."""
    ta, tb, R = 0.7, -0.4, 2.3
    s = pair_cluster([0, 0, 0], [0, 0, R], ti=(-ta / 2, -ta / 2, ta, 0, 0, 0), tj=(-tb / 2, -tb / 2, tb, 0, 0, 0))
    assert energy(s) == pytest.approx(COULOMB * 6 * ta * tb / R ** 5, rel=1e-13)


def test_pair_inside_a_molecule_is_excluded():
    s = pair_cluster([0, 0, 0], [0.3, 0.2, 0.9], qi=0.5, qj=-0.5, di=(0.1, 0, 0), tj=(0.1, -0.1, 0, 0, 0, 0.2),
                     same=True)
    assert energy(s) == 0.0


def test_periodic_exclusion_removes_exactly_the_bare_intramolecular_terms():
    """Splitting the molecules into independent sites adds back each excluded
    pair's bare (cluster) interaction, and nothing else."""
    L = 9.0
    rc, beta, K = small_box_settings(L)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    s = make_waters(8, L, 3)
    split = copy.deepcopy(s)
    split.mol = np.arange(s.n, dtype=np.int32)
    bare = 0.0
    for a, b in itertools.combinations(range(s.n), 2):
        if s.mol[a] == s.mol[b]:
            d = s.xyz[a] - s.xyz[b]
            d -= L * np.rint(d / L)
            bare += energy(pair_cluster(s.xyz[b] + d, s.xyz[b], s.q[a], s.q[b], s.dip[a], s.dip[b],
                                        s.quad[a], s.quad[b]))
    assert energy(split, st) - energy(s, st) == pytest.approx(bare, rel=1e-12)


# ---------------------------------------------------------------- Ewald

@pytest.mark.parametrize("charged", [False, True])
def test_exact_ewald_energy_independent_of_beta(charged):
    """Real + reciprocal + self (+ background) does not depend on the splitting;
    the charged case pins the neutralising-background term."""
    s = make_waters(8, 7.0, 7)
    if charged:
        s.q = s.q.copy()
        s.q[0] += 0.3
    us = [multipole_energy_exact(s, b) for b in (0.45, 0.5446, 0.65)]
    assert max(us) - min(us) < 1e-10 * abs(us[0])


def _lattice(m, a, q, dip):
    pts = np.array(list(itertools.product(range(m), repeat=3)), float)
    n = len(pts)
    return pts, System(xyz=pts * a + 0.1, q=q(pts), dip=np.tile(dip, (n, 1)), quad=np.zeros((n, 6)),
                       alpha=np.ones(n), thole=np.full(n, 0.39), mol=np.arange(n, dtype=np.int32), box=m * a)


def test_rock_salt_madelung_constant():
    """Charges +-1 on a rock-salt lattice (nearest-neighbour distance a): the
    energy per ion pair is -C M / a with the Madelung constant of NaCl,
    M = 1.747564594633182 (standard tables)."""
    a = 2.8
    pts, s = _lattice(4, a, lambda p: np.where(p.sum(1) % 2 == 0, 1.0, -1.0), np.zeros(3))
    for beta in (0.7, 0.9):
        U = multipole_energy_exact(s, beta)
        assert -U / (s.n / 2) * a / COULOMB == pytest.approx(1.747564594633182, rel=1e-12)
    L = s.box
    st = Setup(box=L, cutoff=L / 2 - 1e-6, beta=3.8122 / (L / 2 - 1e-6), grid=32, order=8)
    assert -energy(s, st) / (s.n / 2) * a / COULOMB == pytest.approx(1.747564594633182, rel=1e-6)


def test_cubic_lattice_of_parallel_dipoles():
    """Identical dipoles d on a simple cubic lattice (edge a): the lattice sum
    vanishes by cubic symmetry, so with tin-foil boundary the energy per dipole
    is the surface-term difference, -(2 pi / 3) C |d|^2 / a^3."""
    a, d = 3.0, np.array([0.02, -0.05, 0.03])
    _, s = _lattice(2, a, lambda p: np.zeros(len(p)), d)
    for beta in (0.6, 0.9):
        assert multipole_energy_exact(s, beta) / s.n == pytest.approx(-2 * np.pi / 3 * (d @ d) / a ** 3 * COULOMB,
                                                                      rel=1e-12)


def test_pme_converges_to_exact_ewald():
    """Minimum-image real space + PME approach the lattice sum truncated at the
    same cutoff as the grid is refined, and meet it at order 8."""
    nw = 64
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    s = make_waters(nw, L, 5)
    ue = multipole_energy_exact(s, beta, rmax=rc, nimg=1)
    errs = [abs(energy(s, Setup(box=L, cutoff=rc, beta=beta, grid=k, order=5)) / ue - 1) for k in (24, 32, 48)]
    assert errs[0] > errs[1] > errs[2]
    assert abs(energy(s, Setup(box=L, cutoff=rc, beta=beta, grid=48, order=8)) / ue - 1) < 3e-7


# ---------------------------------------------------------------- gradients

def _box8():
    L = 9.0
    rc, beta, K = small_box_settings(L)
    return make_waters(8, L, 7), Setup(box=L, cutoff=rc, beta=beta, grid=K)


def _shift(s, field, idx, h):
    t = copy.deepcopy(s)
    a = getattr(t, field).copy()
    a[idx] += h
    setattr(t, field, a)
    return t


def _fd(s, st, field, idx, h):
    return (energy(_shift(s, field, idx, h), st) - energy(_shift(s, field, idx, -h), st)) / (2 * h)


@pytest.mark.parametrize("case", ["box8", "cluster"])
def test_forces_match_finite_differences(case):
    if case == "box8":
        s, st = _box8()
    else:
        s, st = make_waters(4, 6.0, 2, periodic=False), Setup.cluster()
    _, F, _, _, _ = multipole_energy(s, st)
    scale = np.abs(F).max()
    for k in (0, 4, 11):
        for a in range(3):
            assert -_fd(s, st, "xyz", (k, a), 1e-5) == pytest.approx(F[k, a], abs=2e-8 * scale)


def test_moment_gradients_match_finite_differences():
    """U is quadratic in the moments, so central differences are exact up to rounding.
    Quadrupoles move along traceless directions only."""
    s, st = _box8()
    _, _, gq, gd, gt = multipole_energy(s, st)
    h = 1e-3
    for k in (1, 6):
        assert _fd(s, st, "q", k, h) == pytest.approx(gq[k], rel=1e-8, abs=1e-9)
        for a in range(3):
            assert _fd(s, st, "dip", (k, a), h) == pytest.approx(gd[k, a], rel=1e-8, abs=1e-9)
        for c in (3, 4, 5):
            assert _fd(s, st, "quad", (k, c), h) == pytest.approx(gt[k, c], rel=1e-8, abs=1e-9)
        # xx - yy (trace kept at zero)
        up = _shift(_shift(s, "quad", (k, 0), h), "quad", (k, 1), -h)
        dn = _shift(_shift(s, "quad", (k, 0), -h), "quad", (k, 1), h)
        assert (energy(up, st) - energy(dn, st)) / (2 * h) == pytest.approx(gt[k, 0] - gt[k, 1], rel=1e-8, abs=1e-9)


def test_euler_identity_and_projection(box648_system):
    """U is homogeneous of degree two in the moments: U = 1/2 sum M . dU/dM.
    The energy and the gradients come from different sums, so this ties them.
    Projected quadrupole gradients have no mean on the diagonal."""
    s, st = box648_system
    U, F, gq, gd, gt = multipole_energy(s, st)
    euler = 0.5 * ((s.q * gq).sum() + (s.dip * gd).sum() + (s.quad * gt).sum())
    assert euler == pytest.approx(U, rel=1e-11)
    assert np.abs(gt[:, :3].sum(1)).max() < 1e-12 * np.abs(gt).max()


def test_rows_match_the_full_evaluation(box648_system):
    s, st = box648_system
    _, F, gq, gd, gt = multipole_energy(s, st)
    rows = np.array([0, 17, 300, 647])
    Fr, gqr, gdr, gtr = multipole_rows(s, st, rows)
    for a, b in ((Fr, F), (gqr, gq), (gdr, gd), (gtr, gt)):
        assert np.allclose(a, b[rows], rtol=1e-11, atol=1e-11 * np.abs(b).max())


def test_cluster_forces_sum_to_zero():
    s = make_waters(5, 8.0, 9, periodic=False)
    _, F, _, _, _ = multipole_energy(s, Setup.cluster())
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).max()


@pytest.fixture(scope="module")
def box648_system():
    w = WATER_648
    return w.system(), Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)

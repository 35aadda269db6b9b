"""Pins of the CPU oracle to closed forms, brute force and physical invariants.

Nothing here compares the oracle with itself: every expected value comes from
a closed form, a library routine, a brute-force definition or an invariant of
the physics (symmetry of T, independence of the Ewald splitting, the
variational energy).
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import Setup
from oracle.energy import polarization_energy, quadratic_form_energy
from oracle.ewald import screened_B, thole_lambdas, thole_x
from oracle.ewald_exact import ExactEwald
from oracle.pairs import brute_force_pairs, periodic_pairs
from oracle.pme import PmeGrid, cardinal_bspline_deriv, dipole_field_recip, permanent_field_recip
from oracle.realspace import multipole_field, multipole_potential, quad_matrix
from oracle.solver import Operator, dense_solve, pcg, rms_debye, solve
from oracle.setup import DEBYE
from paper_1906_01211_gb300.synth import (WATER_648, System, density_box_edge, make_waters,
                                          small_box_settings)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def two_sites(r, alpha=(0.837, 0.496), a=0.39, q=(0.0, 0.0)):
    z = np.zeros((2, 3))
    return System(xyz=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r]]), q=np.array(q, float),
                  dip=z.copy(), quad=np.zeros((2, 6)), alpha=np.array(alpha, float),
                  thole=np.array([a, a]), mol=np.array([0, 1], np.int32), box=None)


@pytest.fixture(scope="module")
def box648():
    w = WATER_648
    s = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    return s, st, Operator(s, st)


@pytest.fixture(scope="module")
def box64():
    nw = 64
    L = density_box_edge(nw)
    rc, beta, K = small_box_settings(L)
    return make_waters(nw, L, 5), L, rc, beta, K


# ---------------------------------------------------------------- pair field

@pytest.mark.parametrize("r", [0.9, 1.6, 2.5, 4.0])
def test_isolated_pair_dipole_field_closed_form(r):
    """Thole-damped field of one dipole along and across the axis.

    By hand from E = -lambda3 mu/r^3 + 3 lambda5 (mu.r) r/r^5:
    along z:  E_z = (2 - 2 e^-x - 3 x e^-x) mu / r^3
    across:   E_x = -(1 - e^-x) mu / r^3,  x = a r^3 / sqrt(a1 a2).
    """
    s = two_sites(r)
    op = Operator(s, Setup.cluster())
    mu = np.zeros((2, 3))
    mu[1] = [0.3, -0.2, 0.7]
    e = op.apply_T(mu)[0]
    x = 0.39 * r ** 3 / math.sqrt(0.837 * 0.496)
    ex = math.exp(-x)
    ez_ref = (2 - 2 * ex - 3 * x * ex) * 0.7 / r ** 3
    ex_ref = -(1 - ex) * 0.3 / r ** 3
    ey_ref = -(1 - ex) * (-0.2) / r ** 3
    assert e == pytest.approx([ex_ref, ey_ref, ez_ref], rel=1e-13, abs=1e-15)


def test_two_site_induced_dipoles_solved_by_hand():
    """2x2 per axis: [1/a1, -t; -t, 1/a2] mu = E, t = axial or transverse coupling."""
    r, a1, a2 = 2.2, 0.837, 0.496
    s = two_sites(r, (a1, a2))
    op = Operator(s, Setup.cluster())
    E0 = np.array([[0.01, -0.02, 0.03], [0.005, 0.015, -0.01]])
    x = 0.39 * r ** 3 / math.sqrt(a1 * a2)
    ex = math.exp(-x)
    t_par = (2 - 2 * ex - 3 * x * ex) / r ** 3
    t_perp = -(1 - ex) / r ** 3
    ref = np.zeros((2, 3))
    for c, t in enumerate((t_perp, t_perp, t_par)):
        det = 1 / (a1 * a2) - t * t
        ref[0, c] = (E0[0, c] / a2 + t * E0[1, c]) / det
        ref[1, c] = (E0[1, c] / a1 + t * E0[0, c]) / det
    mu, it, rms = solve(op, E0, 1e-12)
    assert rms < 1e-12
    assert np.allclose(mu, ref, rtol=1e-10, atol=1e-14)
    assert np.allclose(dense_solve(op.apply_A, E0), ref, rtol=1e-12, atol=1e-15)


def test_thole_lambdas_from_smeared_charge():
    """lambda3 is the charge of the Thole density rho(u) ~ exp(-a u^3) inside r
    (numerical quadrature); lambda5 = lambda3 - (r/3) dlambda3/dr and
    lambda7 = lambda5 - (r/5) dlambda5/dr (finite differences in r)."""
    from scipy.integrate import quad as integrate
    a, aij = 0.39, math.sqrt(0.837 * 0.496)
    norm = 3 * a / (4 * math.pi * aij)

    def lam3_quad(r):
        return integrate(lambda s: 4 * math.pi * s * s * norm * math.exp(-a * s ** 3 / aij), 0, r,
                         epsabs=1e-14, epsrel=1e-13)[0]

    def lam(r, k):
        return thole_lambdas(np.array([thole_x(r, 0.837, 0.496, a, a)]))[k][0]

    h = 1e-5
    for r in (0.5, 1.0, 1.7, 2.6):
        assert lam(r, 0) == pytest.approx(lam3_quad(r), rel=1e-10, abs=1e-13)
        d3 = (lam(r + h, 0) - lam(r - h, 0)) / (2 * h)
        assert lam(r, 1) == pytest.approx(lam(r, 0) - r / 3 * d3, abs=1e-9)
        d5 = (lam(r + h, 1) - lam(r - h, 1)) / (2 * h)
        assert lam(r, 2) == pytest.approx(lam(r, 1) - r / 5 * d5, abs=1e-9)
        d7 = (lam(r + h, 2) - lam(r - h, 2)) / (2 * h)
        assert lam(r, 3) == pytest.approx(lam(r, 2) - r / 7 * d7, abs=1e-9)


def test_screened_kernels_recurrence_is_radial_derivative():
    """dB_n/dr = -r B_{n+1} for the Ewald kernels (checked by finite differences)."""
    r = np.linspace(0.8, 7.0, 13)
    h = 1e-6
    for beta in (0.0, 0.5446):
        B = screened_B(r, beta, 4)
        Bp = screened_B(r + h, beta, 4)
        Bm = screened_B(r - h, beta, 4)
        for n in range(4):
            d = (Bp[n] - Bm[n]) / (2 * h)
            assert np.allclose(d, -r * B[n + 1], rtol=1e-7)


def test_multipole_field_is_minus_gradient_of_potential():
    """E = -grad phi for q, d, Theta with screened kernels (finite differences)."""
    rng = np.random.default_rng(11)
    P = 20
    r = rng.normal(size=(P, 3)) * 2.0
    r *= (2.0 + 3.0 * rng.random(P))[:, None] / np.linalg.norm(r, axis=1)[:, None]
    q = rng.normal(size=P)
    d = rng.normal(size=(P, 3))
    th = rng.normal(size=(P, 6))
    th[:, :3] -= th[:, :3].mean(1, keepdims=True)

    def phi(rr):
        B = screened_B(np.linalg.norm(rr, axis=1), 0.5446, 2)
        return multipole_potential(rr, q, d, th, B[0], B[1], B[2])

    B = screened_B(np.linalg.norm(r, axis=1), 0.5446, 3)
    e = multipole_field(r, q, d, th, B[1], B[2], B[3])
    h = 1e-5
    for a in range(3):
        dv = np.zeros(3)
        dv[a] = h
        fd = -(phi(r + dv) - phi(r - dv)) / (2 * h)
        assert np.allclose(e[:, a], fd, rtol=1e-7, atol=1e-10)


def test_quadrupole_convention_from_point_charges():
    """Buckingham Theta = 1/2 sum q (3 s s - s^2 I) reproduces the exact Coulomb
    field of a small charge cloud far away, to octupole order."""
    rng = np.random.default_rng(3)
    s = rng.normal(size=(6, 3)) * 0.05
    qs = rng.normal(size=6)
    qt = qs.sum()
    d = (qs[:, None] * s).sum(0)
    th = 0.5 * sum(qk * (3 * np.outer(sk, sk) - sk @ sk * np.eye(3)) for qk, sk in zip(qs, s))
    th6 = np.array([th[0, 0], th[1, 1], th[2, 2], th[0, 1], th[0, 2], th[1, 2]])
    for R in (np.array([17.0, -9.0, 21.0]), np.array([-25.0, 4.0, 3.0])):
        diff = R - s
        exact = (qs[:, None] * diff / np.linalg.norm(diff, axis=1)[:, None] ** 3).sum(0)
        B = screened_B(np.array([np.linalg.norm(R)]), 0.0, 3)
        z = np.zeros(1)
        e_qd = multipole_field(R[None], np.array([qt]), d[None], np.zeros((1, 6)), B[1], B[2], B[3])[0]
        e_th = multipole_field(R[None], z, np.zeros((1, 3)), th6[None], B[1], B[2], B[3])[0]
        # the quadrupole term must account for what charge + dipole leave over
        assert np.linalg.norm(exact - e_qd - e_th) < 2e-2 * np.linalg.norm(e_th)


# ---------------------------------------------------------------- pairs

def test_pairs_match_brute_force(box648):
    s, st, _ = box648
    i, j, _ = periodic_pairs(s.xyz, st.box, st.cutoff)
    bi, bj = brute_force_pairs(s.xyz, st.box, st.cutoff)
    assert len(i) == len(bi)
    assert set(zip(i.tolist(), j.tolist())) == set(zip(bi.tolist(), bj.tolist()))


# ---------------------------------------------------------------- symmetry

def test_T_is_symmetric(box648):
    s, st, op = box648
    rng = np.random.default_rng(1)
    m1, m2 = rng.normal(size=(2, s.n, 3)) * 0.1
    for part in range(3):
        a = (m1 * op.apply_T_parts(m2)[part]).sum()
        b = (m2 * op.apply_T_parts(m1)[part]).sum()
        assert abs(a - b) <= 1e-13 * abs(a) + 1e-16
    a = (m1 * op.apply_T(m2)).sum()
    b = (m2 * op.apply_T(m1)).sum()
    assert abs(a - b) <= 1e-13 * abs(a)


# ---------------------------------------------------------------- PME / Ewald

def test_bspline_matches_scipy_basis_element():
    ref = BSpline.basis_element(np.arange(6.0), extrapolate=False)
    u = np.linspace(0.01, 4.99, 97)
    for d in range(4):
        expect = ref.derivative(d)(u) if d else ref(u)
        assert np.allclose(cardinal_bspline_deriv(5, u, d), expect, atol=1e-13)


def test_bspline_moduli_properties():
    """|b(m)|^2 = 1/|sum_k M_n(k+1) exp(2 pi i m k/K)|^2: 1 at m = 0 (the
    B-spline weights sum to one), even in m, and for odd order and even K the
    denominator vanishes at m = K/2, where the neighbour mean is used."""
    from oracle.pme import bspline_moduli, cardinal_bspline
    for K in (16, 24):
        b2 = bspline_moduli(K, 5)
        assert b2[0] == pytest.approx(1.0, abs=1e-14)
        assert np.allclose(b2[1:], b2[1:][::-1], rtol=1e-13)
        kk = np.arange(4)
        den = abs((cardinal_bspline(5, kk + 1.0) * np.exp(2j * np.pi * (K // 2) * kk / K)).sum()) ** 2
        assert den < 1e-12
        assert b2[K // 2] == pytest.approx(0.5 * (b2[K // 2 - 1] + b2[K // 2 + 1]), rel=1e-14)
        assert np.all(np.isfinite(b2)) and np.all(b2 >= 1.0 - 1e-14)


def test_pme_converges_to_kspace_sum(box64):
    s, L, rc, beta, K = box64
    ex = ExactEwald(s, beta)
    rng = np.random.default_rng(0)
    mu = rng.normal(size=(s.n, 3)) * 0.1
    th = quad_matrix(s.quad)
    dip_ex = ex._recip_field(lambda k: -1j * (mu @ k.T))
    perm_ex = ex._recip_field(lambda k: s.q[:, None] - 1j * (s.dip @ k.T)
                              - np.einsum("ma,nab,mb->nm", k, th, k) / 3.0)
    errs = []
    for KK in (24, 32, 48):
        st = Setup(box=L, cutoff=rc, beta=beta, grid=KK, order=5)
        g = PmeGrid(s.xyz, L, KK, 5, beta)
        errs.append((rel(dipole_field_recip(s, st, mu, g), dip_ex),
                     rel(permanent_field_recip(s, st, g), perm_ex)))
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] > errs[1][1] > errs[2][1]
    assert errs[2][0] < 5e-5 and errs[2][1] < 2e-4
    st = Setup(box=L, cutoff=rc, beta=beta, grid=48, order=8)
    g = PmeGrid(s.xyz, L, 48, 8, beta)
    assert rel(dipole_field_recip(s, st, mu, g), dip_ex) < 1e-7
    assert rel(permanent_field_recip(s, st, g), perm_ex) < 1e-7


def _cubic_lattice(m, a, d, alpha):
    pts = np.array([[i, j, k] for i in range(m) for j in range(m) for k in range(m)], float)
    n = len(pts)
    return System(xyz=pts * a + 0.1, q=np.zeros(n), dip=np.tile(d, (n, 1)), quad=np.zeros((n, 6)),
                  alpha=np.full(n, alpha), thole=np.full(n, 0.39), mol=np.arange(n, dtype=np.int32), box=m * a)


def test_cubic_lattice_lorentz_field_and_induced_dipoles():
    """Identical sites with identical permanent dipoles d on a simple cubic
    lattice (edge a). The dipole tensor summed over complete cubic shells
    vanishes, so under tin-foil Ewald the field at every site is the Lorentz
    field k d, k = 4 pi / (3 a^3); the induced dipoles are then uniform with
    mu = alpha k (d + mu), i.e. mu = alpha k d / (1 - alpha k). (Thole damping
    changes the shell sums by x e^-x / r^3 per neighbour, ~1e-14 here.)"""
    a, d, alpha = 3.0, np.array([0.02, -0.05, 0.03]), 0.3
    k = 4 * np.pi / (3 * a ** 3)
    e_ref, mu_ref = k * d, alpha * k * d / (1 - alpha * k)
    s = _cubic_lattice(2, a, d, alpha)
    for beta in (0.8, 1.1):
        ex = ExactEwald(s, beta)
        e0 = ex.permanent_field()
        mu, _, _ = pcg(lambda v: (1 / s.alpha)[:, None] * v - ex.apply_T(v), s.alpha, e0, 1e-13, 100)
        assert np.abs(e0 - e_ref).max() < 1e-12 * np.abs(e_ref).max()
        assert np.abs(mu - mu_ref).max() < 1e-12 * np.abs(mu_ref).max()
    # production oracle (minimum image + PME) on a 3 x 3 x 3 box: complete shells inside the cutoff
    s = _cubic_lattice(3, a, d, alpha)
    rc, beta, K = small_box_settings(s.box)
    errs = []
    for grid, order in ((K, 5), (32, 5), (32, 8)):
        op = Operator(s, Setup(box=s.box, cutoff=rc, beta=beta, grid=grid, order=order))
        e0 = op.permanent_field()
        mu, _, _ = solve(op, e0, 1e-13, 100)
        errs.append((np.abs(e0 - e_ref).max() / np.abs(e_ref).max(), np.abs(mu - mu_ref).max() / np.abs(mu_ref).max()))
    assert errs[0][0] > errs[1][0] > errs[2][0] and errs[2][0] < 1e-5 and errs[2][1] < 1e-5
    # 2 x 2 x 2 box: the neighbours sit at a = L/2, beyond the cutoff, so no
    # pair is listed and reciprocal + self carry the field (the screened
    # nearest-neighbour terms left out are ~3e-5 of it)
    s = _cubic_lattice(2, a, d, alpha)
    rc, beta, K = small_box_settings(s.box)
    op = Operator(s, Setup(box=s.box, cutoff=rc, beta=beta, grid=32, order=8))
    assert op.n_pairs == 0
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-13, 100)
    assert np.abs(e0 - e_ref).max() < 1e-4 * np.abs(e_ref).max()
    assert np.abs(mu - mu_ref).max() < 1e-4 * np.abs(mu_ref).max()


def test_energy_independent_of_ewald_beta():
    """Exact Ewald polarization energy does not depend on the splitting."""
    s = make_waters(8, 7.0, 7)
    us = []
    for beta in (0.45, 0.5446, 0.65):
        ex = ExactEwald(s, beta)
        e0 = ex.permanent_field()
        mu, _, _ = pcg(lambda m: (1 / s.alpha)[:, None] * m - ex.apply_T(m), s.alpha, e0, 1e-12, 500)
        us.append(polarization_energy(mu, e0))
    assert max(us) - min(us) < 1e-8 * abs(us[0])


def test_minimum_image_real_space_equals_lattice_sum_within_cutoff(box64):
    s, L, rc, beta, K = box64
    st = Setup(box=L, cutoff=rc, beta=beta, grid=K)
    op = Operator(s, st)
    ex = ExactEwald(s, beta, rmax=rc, nimg=1)
    rng = np.random.default_rng(4)
    mu = rng.normal(size=(s.n, 3)) * 0.1
    from oracle.realspace import dipole_field, multipole_field as mf, scatter_add
    b1, b2 = ex.mb
    lat_T = scatter_add(s.n, ex.i, dipole_field(ex.r, mu[ex.j], b1, b2))
    p1, p2, p3 = ex.pb
    lat_E = scatter_add(s.n, ex.i, mf(ex.r, s.q[ex.j], s.dip[ex.j], s.quad[ex.j], p1, p2, p3))
    assert rel(op.apply_T_parts(mu)[0], lat_T) < 1e-13
    assert rel(op.permanent_field_parts()[0], lat_E) < 1e-13


def test_production_oracle_matches_exact_ewald(box64):
    """Minimum-image real space + fine PME agree with the exact Ewald sums up to
    the real-space truncation at the cutoff."""
    s, L, rc, beta, K = box64
    ex = ExactEwald(s, beta)
    e_ex = ex.permanent_field()
    mu_ex, _, _ = pcg(lambda m: (1 / s.alpha)[:, None] * m - ex.apply_T(m), s.alpha, e_ex, 1e-12, 500)
    st = Setup(box=L, cutoff=rc, beta=beta, grid=48, order=8)
    op = Operator(s, st)
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-12, 500)
    assert rel(e0, e_ex) < 1e-5
    assert abs(polarization_energy(mu, e0) / polarization_energy(mu_ex, e_ex) - 1) < 1e-6


# ---------------------------------------------------------------- solver / energy

def test_pcg_matches_dense_cholesky(box64):
    s, L, rc, beta, K = box64
    op = Operator(s, Setup(box=L, cutoff=rc, beta=beta, grid=K))
    e0 = op.permanent_field()
    ref = dense_solve(op.apply_A, e0)  # Cholesky: also proves A is SPD here
    tol = 1e-8
    mu, it, rms = solve(op, e0, tol)
    assert rms < tol and it > 3
    assert rms_debye(mu - ref) < 5 * tol


def test_energy_is_variational_minimum(box648):
    s, st, op = box648
    e0 = op.permanent_field()
    mu, _, _ = solve(op, e0, 1e-12)
    u = polarization_energy(mu, e0)
    # the two differ by -C/2 mu.r, first order in the residual r
    assert quadratic_form_energy(op.apply_A, mu, e0) == pytest.approx(u, rel=1e-10)
    # any perturbation raises the quadratic form
    rng = np.random.default_rng(2)
    dmu = rng.normal(size=mu.shape) * 1e-3
    assert quadratic_form_energy(op.apply_A, mu + dmu, e0) > u


def test_rms_is_in_debye():
    z = np.ones((4, 3)) / math.sqrt(3)
    assert rms_debye(z) == pytest.approx(DEBYE)

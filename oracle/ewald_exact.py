"""Direct Ewald lattice sums for tiny periodic boxes (oracle side).

Used to pin the production oracle (minimum-image real space + smooth PME)
against the exact Ewald definition, and to check that the polarization energy
does not depend on the splitting parameter beta. Plain definitions:

real space: sum over all sources j and lattice vectors n (|n| <= nimg) with
    r = x_i - (x_j + n L), r < rmax, skipping (j = i, n = 0); the
    intramolecular exclusion applies only to n = 0 (images of a molecule are
    other molecules);
reciprocal: phi(x) = (1/(pi V)) sum_{m != 0} exp(-pi^2 m~^2/beta^2)/m~^2
    Re[S(m) exp(2 pi i m~ . x)], m~ = m / L,
    S(m) = sum_j rho_j(m) exp(-2 pi i m~ . x_j),
    rho_j(k) = q_j - i k . d_j - (k . Theta_j . k) / 3 with k = 2 pi m~;
    field E = -grad phi = (1/(pi V)) sum f(m) k Im[S exp(i k . x)];
self: +4 beta^3 / (3 sqrt(pi)) times the site's own dipole (tin-foil boundary,
no surface term).
"""
from __future__ import annotations

import itertools

import numpy as np

from .ewald import screened_B, self_field_coefficient, thole_lambdas, thole_x
from .realspace import dipole_field, multipole_field, quad_matrix, scatter_add


def _image_pairs(xyz, L, rmax, nimg):
    n = xyz.shape[0]
    ii, jj, rr, zero = [], [], [], []
    for nv in itertools.product(range(-nimg, nimg + 1), repeat=3):
        shift = np.array(nv, dtype=np.float64) * L
        d = xyz[:, None, :] - (xyz[None, :, :] + shift)
        dist = np.sqrt((d * d).sum(-1))
        mask = dist < rmax
        if nv == (0, 0, 0):
            mask &= ~np.eye(n, dtype=bool)
        a, b = np.nonzero(mask)
        ii.append(a)
        jj.append(b)
        rr.append(d[a, b])
        zero.append(np.full(a.shape, nv == (0, 0, 0)))
    return (np.concatenate(ii), np.concatenate(jj), np.concatenate(rr),
            np.concatenate(zero))


def _kvectors(L, beta, kmax_tol=1e-18):
    mmax = int(np.ceil(beta * L * np.sqrt(-np.log(kmax_tol)) / np.pi)) + 1
    rng = np.arange(-mmax, mmax + 1)
    m = np.array(list(itertools.product(rng, rng, rng)), dtype=np.float64)
    m = m[np.any(m != 0, axis=1)]
    mt = m / L
    m2 = (mt * mt).sum(1)
    f = np.exp(-np.pi ** 2 * m2 / beta ** 2) / m2
    keep = f > kmax_tol * f.max()
    return mt[keep], f[keep]


class ExactEwald:
    """Exact Ewald operator and right-hand side of a tiny periodic system."""

    def __init__(self, sys, beta, rmax=None, nimg=None):
        L = sys.box
        self.sys, self.beta, self.L = sys, beta, L
        if rmax is None:
            rmax = 7.5 / beta  # erfc(7.5) ~ 2.7e-26
        if nimg is None:
            nimg = int(np.ceil(rmax / L)) + 1
        i, j, r, zero = _image_pairs(sys.xyz, L, rmax, nimg)
        dist = np.sqrt((r * r).sum(1))
        self.i, self.j, self.r = i, j, r
        B = screened_B(dist, beta, 3)
        bare = screened_B(dist, 0.0, 3)
        x = thole_x(dist, sys.alpha[i], sys.alpha[j], sys.thole[i], sys.thole[j])
        l3, l5, l7, _ = thole_lambdas(x)
        excluded = zero & (sys.mol[i] == sys.mol[j])
        s = np.where(excluded, 0.0, 1.0)
        self.pb = (B[1] - (1 - s * l3) * bare[1], B[2] - (1 - s * l5) * bare[2],
                   B[3] - (1 - s * l7) * bare[3])
        self.mb = (B[1] - (1 - l3) * bare[1], B[2] - (1 - l5) * bare[2])
        self.mt, self.f = _kvectors(L, beta)
        self.V = L ** 3
        self.selfc = self_field_coefficient(beta)

    def _recip_field(self, rho_fn):
        """Field at every site from sources with structure factor terms rho_j(k)."""
        xyz = self.sys.xyz
        k = 2.0 * np.pi * self.mt                      # (M, 3)
        phase = np.exp(-1j * xyz @ k.T)                # (N, M) exp(-i k.x_j)
        S = (rho_fn(k) * phase).sum(0)                 # (M,)
        t = np.conj(phase) * S[None, :]                # S exp(+i k.x_i)
        return (np.imag(t) * self.f[None, :]) @ k / (np.pi * self.V)

    def permanent_field(self):
        s = self.sys
        b1, b2, b3 = self.pb
        j = self.j
        real = scatter_add(s.n, self.i, multipole_field(self.r, s.q[j], s.dip[j], s.quad[j], b1, b2, b3))
        th = quad_matrix(s.quad)

        def rho(k):
            kth = np.einsum("ma,nab,mb->nm", k, th, k)
            return s.q[:, None] - 1j * (s.dip @ k.T) - kth / 3.0
        return real + self._recip_field(rho) + self.selfc * s.dip

    def apply_T(self, mu):
        s = self.sys
        b1, b2 = self.mb
        real = scatter_add(s.n, self.i, dipole_field(self.r, mu[self.j], b1, b2))

        def rho(k):
            return -1j * (mu @ k.T)
        return real + self._recip_field(rho) + self.selfc * mu


def multipole_energy_exact(sys, beta, rmax=None, nimg=None) -> float:
    """Ewald energy of the permanent multipoles by direct sums (kcal/mol).

    real: 1/2 sum over ordered (i, j, n) of U_ij(x_i - x_j - n L), r < rmax,
    skipping (j = i, n = 0), same-molecule pairs excluded at n = 0 only, with
    U_ij the pair energy of ``multipole`` on the screened kernels;
    reciprocal: (1/(2 pi V)) sum_{m != 0} exp(-pi^2 m~^2/beta^2)/m~^2 |S(m)|^2
    with S(m) = sum_j rho_j(k) exp(-i k.x_j) (rho as above);
    plus the self and neutralising-background terms of ``multipole``.
    """
    from .multipole import _contract, _full, _kernels, _moments, derivative_tensor, self_and_background
    from .setup import COULOMB, Setup

    L = sys.box
    if rmax is None:
        rmax = 7.5 / beta
    if nimg is None:
        nimg = int(np.ceil(rmax / L)) + 1
    i, j, r, zero = _image_pairs(sys.xyz, L, rmax, nimg)
    dist = np.sqrt((r * r).sum(1))
    excl = (zero & (sys.mol[i] == sys.mol[j])).astype(np.float64)
    b = _kernels(dist, excl, beta, 4)
    T = [derivative_tensor(r, b, k) for k in range(5)]
    Mi, Mj = _moments(sys, i), _moments(sys, j)
    u_real = 0.0
    for k in range(3):
        for l in range(3):
            u_real += (-1.0) ** l * float(_full(Mi[k], _contract(T[k + l], Mj[l])).sum())
    u_real *= 0.5
    mt, f = _kvectors(L, beta)
    k = 2.0 * np.pi * mt
    th = quad_matrix(sys.quad)
    rho = sys.q[:, None] - 1j * (sys.dip @ k.T) - np.einsum("ma,nab,mb->nm", k, th, k) / 3.0
    S = (rho * np.exp(-1j * sys.xyz @ k.T)).sum(0)
    u_rec = float((f * np.abs(S) ** 2).sum()) / (2.0 * np.pi * L ** 3)
    u_self = self_and_background(sys, Setup(box=L, beta=beta))[0]
    return COULOMB * (u_real + u_rec + u_self)

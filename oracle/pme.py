"""Smooth particle-mesh Ewald for multipoles and dipoles (oracle side).

The reciprocal-space parts of the permanent field and of T*mu (paper, Section
"Sequential performance": "reciprocal polarization" is part of the measured
polarization time; Section "Conclusion": the reciprocal-space computations
are not yet vectorized). The method is smooth PME (Essmann et al. 1995) with
the multipolar spreading of Sagui, Pedersen & Darden (2004), written out step
by step for a cubic box of edge L and K points per axis, B-spline order n:

1. scaled coordinate u = K x / L (mod K) per axis; for k0 = floor(u), f = u - k0
   the grid points k0 - t (mod K), t = 0..n-1, carry weight M_n(f + t) where
   M_n is the cardinal B-spline on [0, n];
2. spread Q(g) = sum_i (q_i + d_i . grad_i + (1/3) Theta_i : grad_i grad_i) W_i(g),
   W_i(g) = prod_axes M_n, grad_i = (K/L) d/du per axis;
3. phi_grid = inverse DFT (no 1/K^3) of G(m) * forward DFT(Q)(m), with
   G(m) = exp(-pi^2 |m~|^2 / beta^2) / (pi V |m~|^2) * |b(m1) b(m2) b(m3)|^2,
   m~ = m_signed / L, G(0) = 0;
4. field at site i: E_i = -sum_g grad_i W_i(g) phi_grid(g).

|b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2. For odd n and
even K the sum vanishes at m = K/2; there (denominator < 1e-7) |b(m)|^2 is set
to the mean of its neighbours m - 1 and m + 1.
"""
from __future__ import annotations

from math import comb

import numpy as np

from .ewald import self_field_coefficient


def cardinal_bspline(n: int, u: np.ndarray) -> np.ndarray:
    """M_n(u): M_2(u) = max(0, 1 - |u - 1|), M_n = [u M_{n-1}(u) + (n-u) M_{n-1}(u-1)]/(n-1)."""
    u = np.asarray(u, dtype=np.float64)
    if n == 2:
        return np.maximum(0.0, 1.0 - np.abs(u - 1.0))
    return (u * cardinal_bspline(n - 1, u) + (n - u) * cardinal_bspline(n - 1, u - 1.0)) / (n - 1)


def cardinal_bspline_deriv(n: int, u: np.ndarray, d: int) -> np.ndarray:
    """d-th derivative: sum_k (-1)^k C(d, k) M_{n-d}(u - k)  (d <= n - 2)."""
    if d == 0:
        return cardinal_bspline(n, u)
    out = np.zeros_like(np.asarray(u, dtype=np.float64))
    for k in range(d + 1):
        out = out + (-1) ** k * comb(d, k) * cardinal_bspline(n - d, u - k)
    return out


def spline_weights(x: np.ndarray, L: float, K: int, n: int, nderiv: int):
    """Per-axis grid indices and weights.

    x (N,) one Cartesian component. Returns idx (N, n) int and
    w[d] (N, n) = d-th derivative with respect to x (scaled by (K/L)^d).
    """
    u = np.mod(x * (K / L), K)
    u[u >= K] -= K
    k0 = np.floor(u)
    f = u - k0
    t = np.arange(n)
    idx = np.mod(k0[:, None].astype(np.int64) - t[None, :], K)
    arg = f[:, None] + t[None, :]
    s = K / L
    w = [cardinal_bspline_deriv(n, arg, d) * s ** d for d in range(nderiv + 1)]
    return idx, w


def bspline_moduli(K: int, n: int) -> np.ndarray:
    """|b(m)|^2 for m = 0..K-1 with the neighbour-mean rule at a vanishing denominator."""
    kk = np.arange(n - 1)
    mk = cardinal_bspline(n, kk + 1.0)
    m = np.arange(K)
    s = (mk[None, :] * np.exp(2j * np.pi * m[:, None] * kk[None, :] / K)).sum(1)
    den = np.abs(s) ** 2
    b2 = np.full(K, np.nan)
    ok = den >= 1e-7
    b2[ok] = 1.0 / den[ok]
    for k in np.nonzero(~ok)[0]:
        b2[k] = 0.5 * (b2[(k - 1) % K] + b2[(k + 1) % K])
    return b2


def influence(L: float, K: int, n: int, beta: float) -> np.ndarray:
    """G(m) on the half spectrum, shape (K, K, K//2 + 1)."""
    b2 = bspline_moduli(K, n)
    m = np.arange(K)
    ms = np.where(m <= K // 2, m, m - K) / L
    mz = np.arange(K // 2 + 1) / L
    m2 = ms[:, None, None] ** 2 + ms[None, :, None] ** 2 + mz[None, None, :] ** 2
    V = L ** 3
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2)
    g[0, 0, 0] = 0.0
    g = g * b2[:, None, None] * b2[None, :, None] * b2[None, None, :K // 2 + 1]
    return g


class PmeGrid:
    """Spline weights of one set of positions on one grid."""

    def __init__(self, xyz: np.ndarray, L: float, K: int, n: int, beta: float, nderiv: int = 2):
        self.L, self.K, self.n, self.beta = L, K, n, beta
        self.ix, self.wx = spline_weights(xyz[:, 0], L, K, n, nderiv)
        self.iy, self.wy = spline_weights(xyz[:, 1], L, K, n, nderiv)
        self.iz, self.wz = spline_weights(xyz[:, 2], L, K, n, nderiv)
        self.flat = ((self.ix[:, :, None, None] * K + self.iy[:, None, :, None]) * K
                     + self.iz[:, None, None, :]).reshape(xyz.shape[0], -1)
        self.G = influence(L, K, n, beta)

    def _w3(self, dx, dy, dz):
        return np.einsum("pa,pb,pc->pabc", self.wx[dx], self.wy[dy], self.wz[dz])

    def _accumulate(self, blocks: np.ndarray) -> np.ndarray:
        K = self.K
        q = np.bincount(self.flat.ravel(), weights=blocks.reshape(-1), minlength=K ** 3)
        return q.reshape(K, K, K)

    def spread_multipoles(self, q, d, quad6) -> np.ndarray:
        """Q(g) for charges, dipoles and traceless quadrupoles."""
        w = self._w3
        blk = q[:, None, None, None] * w(0, 0, 0)
        blk = blk + d[:, 0, None, None, None] * w(1, 0, 0) \
            + d[:, 1, None, None, None] * w(0, 1, 0) + d[:, 2, None, None, None] * w(0, 0, 1)
        t = quad6
        quad = (t[:, 0, None, None, None] * w(2, 0, 0) + t[:, 1, None, None, None] * w(0, 2, 0)
                + t[:, 2, None, None, None] * w(0, 0, 2)
                + 2.0 * t[:, 3, None, None, None] * w(1, 1, 0)
                + 2.0 * t[:, 4, None, None, None] * w(1, 0, 1)
                + 2.0 * t[:, 5, None, None, None] * w(0, 1, 1))
        return self._accumulate(blk + quad / 3.0)

    def spread_dipoles(self, mu) -> np.ndarray:
        """Q(g) for point dipoles mu (N, 3)."""
        w = self._w3
        blk = mu[:, 0, None, None, None] * w(1, 0, 0) + mu[:, 1, None, None, None] * w(0, 1, 0) \
            + mu[:, 2, None, None, None] * w(0, 0, 1)
        return self._accumulate(blk)

    def convolve(self, Q: np.ndarray) -> np.ndarray:
        """phi_grid = unnormalised inverse DFT of G * forward DFT(Q)."""
        K = self.K
        F = np.fft.rfftn(Q)
        return np.fft.irfftn(F * self.G, s=(K, K, K), axes=(0, 1, 2), norm="forward")

    def gather_field(self, phi: np.ndarray) -> np.ndarray:
        """E_i = -sum_g grad_i W_i(g) phi(g)."""
        vals = phi.reshape(-1)[self.flat].reshape(-1, self.n, self.n, self.n)
        ex = np.einsum("pabc,pabc->p", self._w3(1, 0, 0), vals)
        ey = np.einsum("pabc,pabc->p", self._w3(0, 1, 0), vals)
        ez = np.einsum("pabc,pabc->p", self._w3(0, 0, 1), vals)
        return -np.stack([ex, ey, ez], axis=1)

    def gather_potential(self, phi: np.ndarray) -> np.ndarray:
        vals = phi.reshape(-1)[self.flat].reshape(-1, self.n, self.n, self.n)
        return np.einsum("pabc,pabc->p", self._w3(0, 0, 0), vals)


def permanent_field_recip(sys, setup, grid: PmeGrid | None = None) -> np.ndarray:
    """Reciprocal-space permanent field (no self term), (N, 3)."""
    g = grid or PmeGrid(sys.xyz, setup.box, setup.grid, setup.order, setup.beta)
    return g.gather_field(g.convolve(g.spread_multipoles(sys.q, sys.dip, sys.quad)))


def dipole_field_recip(sys, setup, mu, grid: PmeGrid | None = None) -> np.ndarray:
    """Reciprocal-space part of T*mu (no self term); mu (N, 3) or (N, 3, nb)."""
    g = grid or PmeGrid(sys.xyz, setup.box, setup.grid, setup.order, setup.beta)
    if mu.ndim == 3:
        return np.stack([dipole_field_recip(sys, setup, mu[:, :, b], g)
                         for b in range(mu.shape[2])], axis=2)
    return g.gather_field(g.convolve(g.spread_dipoles(mu)))


def self_field(setup, dip) -> np.ndarray:
    """Ewald self field +4 beta^3/(3 sqrt(pi)) * dipole of the site itself."""
    if not setup.periodic:
        return np.zeros_like(dip)
    return self_field_coefficient(setup.beta) * dip

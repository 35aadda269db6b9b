"""Operator, PCG solve and dense reference solve (oracle side).

Problem (the polarization equation whose right-hand side is computed by
``efld0_direct2`` and whose operator is applied by ``tmatxb_pme2``, paper
Section "Hotspots"):

    A mu = E0,   A = diag(1/alpha) - T,   T = T_real + T_recip + T_self,
    E0 = E0_real + E0_recip + E0_self.

The paper names only "the convergence method"; the solver here is conjugate
gradients with the diagonal preconditioner M = diag(alpha) (Saad, Iterative
Methods for Sparse Linear Systems, Algorithm 9.1), written in the order:

    mu_0 = alpha E0 (or a supplied guess);  r_0 = E0 - A mu_0;  z_0 = alpha r_0;  p_0 = z_0
    repeat:  q = A p;  gamma = (r.z)/(p.q);  mu += gamma p;  r -= gamma q;
             z = alpha r;  stop if RMS_D(z) < tol;
             beta = (r.z)_new/(r.z)_old;  p = z + beta p
    RMS_D(z) = DEBYE * sqrt(sum_i |z_i|^2 / N)   (Debye)
"""
from __future__ import annotations

import numpy as np

from .pairs import pairs_for
from .pme import PmeGrid, dipole_field_recip, permanent_field_recip, self_field
from .realspace import PairTerms, dipole_field_real, permanent_field_real
from .setup import DEBYE


class Operator:
    """E0 and T*mu for one system and Setup, with geometry terms cached."""

    def __init__(self, sys, setup):
        self.sys, self.setup = sys, setup
        i, j, r = pairs_for(sys.xyz, setup)
        self.terms = PairTerms(sys, setup, i, j, r)
        self.grid = None
        if setup.periodic:
            self.grid = PmeGrid(sys.xyz, setup.box, setup.grid, setup.order, setup.beta)

    @property
    def n_pairs(self) -> int:
        return int(self.terms.i.shape[0])

    def permanent_field(self) -> np.ndarray:
        s = self.sys
        e = permanent_field_real(s, self.setup, self.terms)
        if self.setup.periodic:
            e = e + permanent_field_recip(s, self.setup, self.grid) + self_field(self.setup, s.dip)
        return e

    def permanent_field_parts(self):
        s = self.sys
        real = permanent_field_real(s, self.setup, self.terms)
        if not self.setup.periodic:
            return real, np.zeros_like(real), np.zeros_like(real)
        return real, permanent_field_recip(s, self.setup, self.grid), self_field(self.setup, s.dip)

    def apply_T(self, mu: np.ndarray) -> np.ndarray:
        t = dipole_field_real(self.sys, self.setup, mu, self.terms)
        if self.setup.periodic:
            t = t + dipole_field_recip(self.sys, self.setup, mu, self.grid) + self_field(self.setup, mu)
        return t

    def apply_T_parts(self, mu):
        real = dipole_field_real(self.sys, self.setup, mu, self.terms)
        if not self.setup.periodic:
            return real, np.zeros_like(real), np.zeros_like(real)
        return real, dipole_field_recip(self.sys, self.setup, mu, self.grid), self_field(self.setup, mu)

    def apply_A(self, mu: np.ndarray) -> np.ndarray:
        a = self.sys.alpha
        inv = (1.0 / a)[:, None] if mu.ndim == 2 else (1.0 / a)[:, None, None]
        return inv * mu - self.apply_T(mu)


def rms_debye(z: np.ndarray) -> float:
    return float(DEBYE * np.sqrt((z * z).sum() / z.shape[0]))


def pcg(apply_A, alpha, E0, tol_debye, max_iter=100, mu0=None):
    """Diagonal-preconditioned CG. Returns (mu, iterations, final RMS in Debye).

    Raises if p.Ap <= 0 (the operator would not be positive definite) and
    returns converged=False through the iteration count reaching max_iter.
    """
    a = alpha[:, None]
    mu = a * E0 if mu0 is None else mu0.copy()
    r = E0 - apply_A(mu)
    z = a * r
    rms = rms_debye(z)
    if rms < tol_debye:
        return mu, 0, rms
    p = z.copy()
    rz = float((r * z).sum())
    for it in range(1, max_iter + 1):
        q = apply_A(p)
        pq = float((p * q).sum())
        if not pq > 0.0:
            raise ArithmeticError("p.Ap <= 0: operator not positive definite")
        gamma = rz / pq
        mu = mu + gamma * p
        r = r - gamma * q
        z = a * r
        rms = rms_debye(z)
        if rms < tol_debye:
            return mu, it, rms
        rz_new = float((r * z).sum())
        p = z + (rz_new / rz) * p
        rz = rz_new
    return mu, max_iter, rms


def solve(op: Operator, E0: np.ndarray, tol_debye: float, max_iter: int = 100, mu0=None):
    return pcg(op.apply_A, op.sys.alpha, E0, tol_debye, max_iter, mu0)


def dense_matrix(apply_A, n: int, batch: int = 96) -> np.ndarray:
    """Assemble the 3N x 3N matrix of a linear operator column by column."""
    m = 3 * n
    A = np.empty((m, m))
    for c0 in range(0, m, batch):
        cols = range(c0, min(m, c0 + batch))
        E = np.zeros((n, 3, len(cols)))
        for k, c in enumerate(cols):
            E[c // 3, c % 3, k] = 1.0
        out = apply_A(E)
        A[:, c0:c0 + len(cols)] = out.reshape(m, len(cols))
    return A


def dense_solve(apply_A, E0: np.ndarray) -> np.ndarray:
    """Cholesky solve of the assembled operator (raises if not SPD)."""
    n = E0.shape[0]
    A = dense_matrix(apply_A, n)
    A = 0.5 * (A + A.T)
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, E0.reshape(-1))
    return np.linalg.solve(L.T, y).reshape(n, 3)

"""Divide-and-conquer Jacobi iterations (DC-JI) (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's outlook (Section "Perspectives on Tinker-HP 1.2 performance")
names DC-JI (Nocito & Beran, 2018) as the polarization solver of the outer
level of its multi-timestep integrator. Reading used here: the sites are
split into blocks of whole molecules (by a regular grid of cells over the box,
each molecule going to the cell of its first site); every iteration solves
each block's own equations exactly, with the other blocks' dipoles taken from
the previous iteration,

    A_BB mu_B^(k+1) = E_B - sum_{C != B} A_BC mu_C^(k),    mu^(0) = alpha E,

and stops when the RMS (Debye) of the preconditioned residual alpha (E - A mu)
is below the tolerance, the criterion of ``solver``. The operator is
assembled densely (3N columns of A), so this is for small systems; the
extrapolation the method's authors add to the iteration is left out.
"""
from __future__ import annotations

import numpy as np

from .solver import dense_matrix, rms_debye


def cell_blocks(sys, cells_per_axis: int):
    """Blocks of whole molecules: list of site-index arrays (empty cells dropped)."""
    L = sys.box if sys.box is not None else float(np.ptp(sys.xyz, axis=0).max()) + 1e-9
    lo = sys.xyz.min(axis=0) if sys.box is None else np.zeros(3)
    first = {}
    for a, m in enumerate(sys.mol):
        first.setdefault(int(m), a)
    key = {}
    for m, a in first.items():
        u = (sys.xyz[a] - lo) / L
        u = u - np.floor(u) if sys.box is not None else u
        c = np.minimum((u * cells_per_axis).astype(int), cells_per_axis - 1)
        key[m] = (c[0] * cells_per_axis + c[1]) * cells_per_axis + c[2]
    cells = {}
    for a, m in enumerate(sys.mol):
        cells.setdefault(key[int(m)], []).append(a)
    return [np.array(v, dtype=np.int64) for _, v in sorted(cells.items())]


def dcji(op, blocks, tol_debye: float, max_iter: int = 200, A=None):
    """(mu, iterations, final RMS in Debye) of block-Jacobi iterations on A mu = E."""
    sys = op.sys
    n = sys.n
    E = op.permanent_field()
    if A is None:
        A = dense_matrix(op.apply_A, n)
    e = E.reshape(-1)
    idx = [np.stack([3 * b, 3 * b + 1, 3 * b + 2], axis=1).reshape(-1) for b in blocks]
    chol = [np.linalg.cholesky(0.5 * (A[np.ix_(k, k)] + A[np.ix_(k, k)].T)) for k in idx]
    mu = (sys.alpha[:, None] * E).reshape(-1)
    al = np.repeat(sys.alpha, 3)

    def rms(m):
        return rms_debye((al * (e - A @ m)).reshape(n, 3))

    r = rms(mu)
    it = 0
    while r >= tol_debye and it < max_iter:
        new = mu.copy()
        for k, L in zip(idx, chol):
            rhs = e[k] - A[k] @ mu + A[np.ix_(k, k)] @ mu[k]
            new[k] = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
        mu = new
        it += 1
        r = rms(mu)
    return mu.reshape(n, 3), it, r

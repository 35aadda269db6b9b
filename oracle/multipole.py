"""Permanent-multipole energy and its gradients (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

Besides the polarization routines, the paper's profile of an AMOEBA step
(Section "Hotspots") lists the interaction of the permanent multipoles with
each other (``empole1``: energy and forces) as the other large electrostatic
cost. Here the multipoles are charges, dipoles and traceless (Buckingham)
quadrupoles fixed in the global frame, so there are no torques.

Pair energy. For sites i, j with r = x_i - x_j and a radial kernel B_0(|r|),
the energy of i's multipole in the potential of j's is

    U_ij = (q_i + d_i.grad + 1/3 Theta_i:grad grad)
           (q_j - d_j.grad + 1/3 Theta_j:grad grad) B_0,     grad acting on r,

the potential of j being phi_j = q_j B_0 + (d_j.r) B_1 + 1/3 (r.Theta_j.r) B_2.
With grad B_n = -r B_{n+1}, the n-th derivative tensor of B_0 is

    T^(n)_{a1..an} = sum_m (-1)^(n-m) B_{n-m} sum over the ways of choosing m
                     disjoint index pairs of  prod delta_{pair} prod r_{other}

(every derivative either lowers the kernel, giving -r, or turns an earlier r
into a delta). With the moment tensors M^(0) = q, M^(1) = d, M^(2) = Theta/3,
U_ij = sum_{k,l} (-1)^l <M_i^(k) (x) M_j^(l), T^(k+l)>. The potential
derivatives ("jet") of j at i are J^(k) = sum_l (-1)^l T^(k+l) . M_j^(l), so
U_ij = sum_k <M_i^(k), J^(k)> and the force on i is -sum_k <M_i^(k), J^(k+1)>.
Kernels: the Ewald-screened B_n, and for two sites of one molecule B_n - bare_n
(the pair is excluded: the full bare term is removed). No Thole damping: that
belongs to polarization only.

Total (Ewald sum, tin-foil boundary), in kcal/mol through C:

    U = C [ sum over unique pairs within the cutoff of U_ij     (minimum image)
          + 1/2 sum_g Q(g) phi_grid(g)                          (smooth PME)
          - beta/sqrt(pi) sum_i (q_i^2 + 2 beta^2/3 |d_i|^2
                                 + 8 beta^4/45 Theta_i:Theta_i)  (self)
          - pi Q_tot^2 / (2 V beta^2) ]                          (background)

with Q the multipole spread and phi_grid its convolution (``pme``). The self
term is minus half of each site's interaction with its own erf kernel
erf(beta r)/r at r -> 0, whose derivative kernels there are
(2 beta/sqrt(pi)) (2 beta^2)^n / (2n + 1). The background term is the k = 0
limit for a net charge Q_tot (zero for neutral systems). An isolated cluster
(no box) has only the pair sum, over all pairs, with bare kernels.

Gradients: F_k = -dU/dx_k; dU/dq_k = C phi_k, dU/dd_k = C grad phi_k and, per
matrix entry, dU/dTheta_k,ab = C/3 (grad grad phi_k)_ab, phi the total
potential of the other multipoles at k (with the self and background parts).
Quadrupole gradients are returned for the six stored numbers (xx, yy, zz, xy,
xz, yz; each off-diagonal stands for two entries, so it gets twice the entry
derivative) and projected onto traceless changes: the mean of the three
diagonal gradients is removed. That makes them unique: the trace of Theta is
fixed at zero, so any equal shift of the diagonal gradients has no meaning.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

from .ewald import SQRT_PI, screened_B
from .pairs import cluster_pairs, minimum_image, periodic_pairs
from .pme import PmeGrid
from .realspace import quad_matrix, scatter_add
from .setup import COULOMB

_LET = "abcdefgh"
_CHUNK = 20000


@lru_cache(maxsize=None)
def _pairings(n: int):
    """Every way to pick disjoint index pairs among positions 0..n-1.

    Returns a tuple of (pairs, singles); n = 5 gives 1 + 10 + 15 = 26 entries.
    """
    out = []

    def rec(pos, free, pairs, singles):
        if pos == n:
            out.append((tuple(pairs), tuple(singles)))
            return
        if pos not in free:
            rec(pos + 1, free, pairs, singles)
            return
        rec(pos + 1, free - {pos}, pairs, singles + [pos])
        for q in sorted(free):
            if q > pos:
                rec(pos + 1, free - {pos, q}, pairs + [(pos, q)], singles)

    rec(0, frozenset(range(n)), [], [])
    return tuple(out)


def derivative_tensor(r: np.ndarray, B, n: int) -> np.ndarray:
    """T^(n) = grad^n B_0 at displacements r (P, 3): shape (P,) + (3,) * n."""
    P = r.shape[0]
    T = np.zeros((P,) + (3,) * n)
    for idx in itertools.product(range(3), repeat=n):
        acc = np.zeros(P)
        for pairs, singles in _pairings(n):
            if any(idx[a] != idx[b] for a, b in pairs):
                continue
            term = (-1.0) ** (n - len(pairs)) * B[n - len(pairs)]
            for s in singles:
                term = term * r[:, idx[s]]
            acc = acc + term
        T[(slice(None),) + idx] = acc
    return T


def _contract(T: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Contract the leading indices of T (P, 3^n) with a rank-k moment A (P, 3^k)."""
    k, n = A.ndim - 1, T.ndim - 1
    sa, st, so = "p" + _LET[:k], "p" + _LET[:n], "p" + _LET[k:n]
    return np.einsum(f"{sa},{st}->{so}", A, T)


def _moments(sys, idx):
    return [sys.q[idx], sys.dip[idx], quad_matrix(sys.quad[idx]) / 3.0]


def _jets(T, M, sign_k: bool):
    """J^(k), k = 0..3, of sources with moments M through tensors T^(0..5).

    J^(k) = sum_l (-1)^l T^(k+l).M^(l): the potential derivatives at the field
    point. For the reversed displacement (sign_k), T^(n)(-r) = (-1)^n T^(n)(r)
    gives J^(k) = (-1)^k sum_l T^(k+l).M^(l).
    """
    out = []
    for k in range(4):
        acc = 0.0
        for l in range(3):
            s = 1.0 if sign_k else (-1.0) ** l
            acc = acc + s * _contract(T[k + l], M[l])
        out.append(acc * ((-1.0) ** k if sign_k else 1.0))
    return out


def _full(A, J):
    """<A, J> over all indices, per pair."""
    return (A.reshape(A.shape[0], -1) * J.reshape(J.shape[0], -1)).sum(1)


def _store6(G: np.ndarray) -> np.ndarray:
    """(N, 3, 3) entry derivatives -> six stored numbers, off-diagonals doubled."""
    return np.stack([G[:, 0, 0], G[:, 1, 1], G[:, 2, 2],
                     2.0 * G[:, 0, 1], 2.0 * G[:, 0, 2], 2.0 * G[:, 1, 2]], axis=1)


def project_traceless(gt6: np.ndarray) -> np.ndarray:
    """Remove the mean of the three diagonal gradients (traceless changes only)."""
    out = np.array(gt6, dtype=np.float64, copy=True)
    out[:, :3] -= out[:, :3].mean(axis=1, keepdims=True)
    return out


def _pair_list(sys, setup):
    if setup.periodic:
        return periodic_pairs(sys.xyz, setup.box, setup.cutoff)
    return cluster_pairs(sys.xyz)


def _kernels(dist, excluded, beta, nmax):
    """[b_0..b_nmax]: screened B_n, minus bare_n for excluded pairs."""
    B = screened_B(dist, beta, nmax)
    bare = screened_B(dist, 0.0, nmax)
    return [b - excluded * e for b, e in zip(B, bare)]


def real_space(sys, setup, pairs=None):
    """Pair-sum part: (U/C, force/C (N,3), phi (N,), grad phi (N,3), grad grad phi (N,3,3))."""
    n = sys.n
    i_all, j_all, r_all = pairs if pairs is not None else _pair_list(sys, setup)
    beta = setup.beta if setup.periodic else 0.0
    U = 0.0
    F = np.zeros((n, 3))
    phi = np.zeros(n)
    g1 = np.zeros((n, 3))
    g2 = np.zeros((n, 3, 3))
    for a in range(0, len(i_all), _CHUNK):
        i, j, r = i_all[a:a + _CHUNK], j_all[a:a + _CHUNK], r_all[a:a + _CHUNK]
        dist = np.sqrt(np.einsum("pa,pa->p", r, r))
        excl = (sys.mol[i] == sys.mol[j]).astype(np.float64)
        B = _kernels(dist, excl, beta, 5)
        T = [derivative_tensor(r, B, k) for k in range(6)]
        Mi, Mj = _moments(sys, i), _moments(sys, j)
        Ji = _jets(T, Mj, sign_k=False)   # potential of j at i, r = x_i - x_j
        Jj = _jets(T, Mi, sign_k=True)    # potential of i at j, displacement -r
        U += float(sum(_full(Mi[k], Ji[k]) for k in range(3)).sum())
        fi = -sum(_contract(Ji[k + 1], Mi[k]) for k in range(3))
        F += scatter_add(n, i, fi) - scatter_add(n, j, fi)
        phi += np.bincount(i, Ji[0], minlength=n) + np.bincount(j, Jj[0], minlength=n)
        g1 += scatter_add(n, i, Ji[1]) + scatter_add(n, j, Jj[1])
        g2 += scatter_add(n, i, Ji[2]) + scatter_add(n, j, Jj[2])
    return U, F, phi, g1, g2


def reciprocal(sys, setup, grid: PmeGrid | None = None):
    """Smooth-PME part: (U/C, force/C, phi, grad phi, grad grad phi)."""
    g = grid if grid is not None and len(grid.wx) > 3 else PmeGrid(
        sys.xyz, setup.box, setup.grid, setup.order, setup.beta, nderiv=3)
    Q = g.spread_multipoles(sys.q, sys.dip, sys.quad)
    phig = g.convolve(Q)
    U = 0.5 * float((Q * phig).sum())
    vals = phig.reshape(-1)[g.flat].reshape(-1, g.n, g.n, g.n)

    def deriv(*axes):
        o = [0, 0, 0]
        for a in axes:
            o[a] += 1
        return np.einsum("pa,pb,pc,pabc->p", g.wx[o[0]], g.wy[o[1]], g.wz[o[2]], vals)

    n = sys.n
    phi = deriv()
    g1 = np.stack([deriv(a) for a in range(3)], 1)
    g2 = np.empty((n, 3, 3))
    g3 = np.empty((n, 3, 3, 3))
    for a in range(3):
        for b in range(3):
            g2[:, a, b] = deriv(a, b)
            for c in range(3):
                g3[:, a, b, c] = deriv(a, b, c)
    th = quad_matrix(sys.quad) / 3.0
    F = -(sys.q[:, None] * g1 + np.einsum("pb,pba->pa", sys.dip, g2)
          + np.einsum("pbc,pbca->pa", th, g3))
    return U, F, phi, g1, g2


def self_and_background(sys, setup):
    """Self and neutralising-background parts: (U/C, phi, grad phi, grad grad phi)."""
    beta, V = setup.beta, setup.box ** 3
    th = quad_matrix(sys.quad)
    thth = np.einsum("pab,pab->p", th, th)
    dd = np.einsum("pa,pa->p", sys.dip, sys.dip)
    qtot = float(sys.q.sum())
    U = -beta / SQRT_PI * float((sys.q ** 2 + 2.0 * beta ** 2 / 3.0 * dd
                                 + 8.0 * beta ** 4 / 45.0 * thth).sum())
    U -= np.pi * qtot ** 2 / (2.0 * V * beta ** 2)
    c = 2.0 * beta / SQRT_PI
    phi = -c * sys.q - np.pi * qtot / (V * beta ** 2)
    g1 = -c * (2.0 * beta ** 2 / 3.0) * sys.dip
    # dU/dTheta_ab = C/3 g2_ab must equal -C c (8 beta^4/45) Theta_ab
    g2 = -c * (8.0 * beta ** 4 / 15.0) * th
    return U, phi, g1, g2


def multipole_energy(sys, setup, with_gradients: bool = True):
    """U (kcal/mol) and, if asked, (F, dU/dq, dU/dd, dU/dTheta6 projected)."""
    U, F, phi, g1, g2 = real_space(sys, setup)
    if setup.periodic:
        Ur, Fr, phr, g1r, g2r = reciprocal(sys, setup)
        Us, phs, g1s, g2s = self_and_background(sys, setup)
        U, F = U + Ur + Us, F + Fr
        phi, g1, g2 = phi + phr + phs, g1 + g1r + g1s, g2 + g2r + g2s
    U *= COULOMB
    if not with_gradients:
        return U
    gt = project_traceless(_store6(COULOMB * g2 / 3.0))
    return U, COULOMB * F, COULOMB * phi, COULOMB * g1, gt


def multipole_rows(sys, setup, rows, grid: PmeGrid | None = None):
    """(F, dU/dq, dU/dd, dU/dTheta6 projected) at the given sites only.

    Real space by a direct scan of each row's neighbours; reciprocal space from
    the full grid. For checking large systems at sampled atoms.
    """
    rows = np.asarray(rows, dtype=np.int64)
    m = len(rows)
    F = np.zeros((m, 3))
    phi = np.zeros(m)
    g1 = np.zeros((m, 3))
    g2 = np.zeros((m, 3, 3))
    beta = setup.beta if setup.periodic else 0.0
    for k, a in enumerate(rows):
        others = np.concatenate([np.arange(a), np.arange(a + 1, sys.n)])
        r = minimum_image(sys.xyz[a] - sys.xyz[others], setup.box if setup.periodic else None)
        if setup.periodic:
            keep = np.einsum("pa,pa->p", r, r) < setup.cutoff ** 2
            others, r = others[keep], r[keep]
        ii = np.full(others.shape, a, dtype=np.int64)
        dist = np.sqrt(np.einsum("pa,pa->p", r, r))
        excl = (sys.mol[ii] == sys.mol[others]).astype(np.float64)
        B = _kernels(dist, excl, beta, 5)
        T = [derivative_tensor(r, B, n) for n in range(6)]
        Ji = _jets(T, _moments(sys, others), sign_k=False)
        Mi = _moments(sys, ii)
        F[k] = (-sum(_contract(Ji[n + 1], Mi[n]) for n in range(3))).sum(0)
        phi[k], g1[k], g2[k] = Ji[0].sum(), Ji[1].sum(0), Ji[2].sum(0)
    if setup.periodic:
        _, Fr, phr, g1r, g2r = reciprocal(sys, setup, grid)
        _, phs, g1s, g2s = self_and_background(sys, setup)
        F += Fr[rows]
        phi += phr[rows] + phs[rows]
        g1 += g1r[rows] + g1s[rows]
        g2 += g2r[rows] + g2s[rows]
    gt = project_traceless(_store6(COULOMB * g2 / 3.0))
    return COULOMB * F, COULOMB * phi, COULOMB * g1, gt


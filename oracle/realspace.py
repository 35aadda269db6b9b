"""Real-space pair sums (oracle side).

Right-hand side: the permanent-multipole field at each polarizable site
(paper, Section "Hotspots": ``efld0_direct2`` computes the right-hand side of
the polarization equation). Operator: the dipole field T*mu (paper, Section
"Hotspots": ``tmatxb_pme2`` is the matrix-vector product applied at each
solver iteration). Both are sums over neighbour pairs within the cutoff.

For field point i and source j, r = x_i - x_j (minimum image), r = |r|:

  potential of a multipole (q, d, Theta) (Buckingham traceless Theta):
      phi = q B0 + (d.r) B1 + (1/3) (r.Theta.r) B2
  field E = -grad phi:
      E = q B1 r - B1 d + B2 (d.r) r - (2/3) B2 Theta r + (1/3) B3 (r.Theta.r) r
  dipole field (mutual induction):
      E = -B1u mu + B2u (mu.r) r

Damped coefficients (Thole, AMOEBA): B_n^eff = B_n - (1 - s lambda_{2n+1}) bare_n.
Permanent field: s = 0 for two sites of the same molecule (the pair is
excluded; under Ewald the screened term minus the full bare term remains),
s = 1 otherwise. Mutual induction: s = 1 for every pair (intramolecular
mutual induction is kept). With beta = 0 (clusters) B_n = bare_n.
"""
from __future__ import annotations

import numpy as np

from .ewald import screened_B, thole_lambdas, thole_x
from .pairs import minimum_image, pairs_for


def quad_matrix(quad6: np.ndarray) -> np.ndarray:
    """(..., 6) [xx, yy, zz, xy, xz, yz] -> (..., 3, 3) symmetric matrix."""
    q = np.asarray(quad6)
    m = np.empty(q.shape[:-1] + (3, 3))
    m[..., 0, 0] = q[..., 0]
    m[..., 1, 1] = q[..., 1]
    m[..., 2, 2] = q[..., 2]
    m[..., 0, 1] = m[..., 1, 0] = q[..., 3]
    m[..., 0, 2] = m[..., 2, 0] = q[..., 4]
    m[..., 1, 2] = m[..., 2, 1] = q[..., 5]
    return m


def scatter_add(n: int, idx: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """out[k] = sum of vals[p] over p with idx[p] == k; vals (P, ...)."""
    flat = vals.reshape(vals.shape[0], int(np.prod(vals.shape[1:])))
    out = np.empty((n, flat.shape[1]))
    for c in range(flat.shape[1]):
        out[:, c] = np.bincount(idx, weights=flat[:, c], minlength=n)
    return out.reshape((n,) + vals.shape[1:])


class PairTerms:
    """Distances, screened/bare kernels and Thole factors of a pair list."""

    def __init__(self, sys, setup, i, j, r):
        self.i, self.j, self.r = i, j, r
        self.dist = np.sqrt(np.einsum("pa,pa->p", r, r))
        beta = setup.beta if setup.periodic else 0.0
        self.B = screened_B(self.dist, beta, 4)
        self.bare = screened_B(self.dist, 0.0, 4)
        x = thole_x(self.dist, sys.alpha[i], sys.alpha[j], sys.thole[i], sys.thole[j])
        self.x = x
        self.lam = thole_lambdas(x)  # l3, l5, l7, l9
        self.inter = (sys.mol[i] != sys.mol[j]).astype(np.float64)

    def permanent_coeffs(self):
        """(B1, B2, B3) damped and with the intramolecular exclusion."""
        s = self.inter
        l3, l5, l7, _ = self.lam
        b1 = self.B[1] - (1.0 - s * l3) * self.bare[1]
        b2 = self.B[2] - (1.0 - s * l5) * self.bare[2]
        b3 = self.B[3] - (1.0 - s * l7) * self.bare[3]
        return b1, b2, b3

    def mutual_coeffs(self):
        """(B1u, B2u): damped kernels of the dipole-dipole tensor."""
        l3, l5, _, _ = self.lam
        b1 = self.B[1] - (1.0 - l3) * self.bare[1]
        b2 = self.B[2] - (1.0 - l5) * self.bare[2]
        return b1, b2


def multipole_field(r, q, d, quad6, b1, b2, b3):
    """Field at displacement r (field point minus source) of multipoles."""
    th = quad_matrix(quad6)
    thr = np.einsum("pab,pb->pa", th, r)
    rthr = np.einsum("pa,pa->p", r, thr)
    dr = np.einsum("pa,pa->p", d, r)
    radial = q * b1 + b2 * dr + b3 * rthr / 3.0
    return radial[:, None] * r - b1[:, None] * d - (2.0 / 3.0) * b2[:, None] * thr


def multipole_potential(r, q, d, quad6, b0, b1, b2):
    """Potential at displacement r of multipoles: q B0 + (d.r) B1 + (r.Th.r) B2 / 3."""
    th = quad_matrix(quad6)
    rthr = np.einsum("pa,pab,pb->p", r, th, r)
    return q * b0 + np.einsum("pa,pa->p", d, r) * b1 + rthr * b2 / 3.0


def dipole_field(r, mu, b1u, b2u):
    """Field at displacement r of point dipoles mu: -B1u mu + B2u (mu.r) r.

    mu may carry a trailing batch axis: (P, 3) or (P, 3, nb).
    """
    if mu.ndim == 2:
        mr = np.einsum("pa,pa->p", mu, r)
        return -b1u[:, None] * mu + (b2u * mr)[:, None] * r
    mr = np.einsum("pab,pa->pb", mu, r)
    return -b1u[:, None, None] * mu + b2u[:, None, None] * mr[:, None, :] * r[:, :, None]


def pair_terms(sys, setup, pairs=None) -> PairTerms:
    if pairs is None:
        pairs = pairs_for(sys.xyz, setup)
    i, j, r = pairs
    return PairTerms(sys, setup, i, j, r)


def permanent_field_real(sys, setup, terms: PairTerms | None = None) -> np.ndarray:
    """Real-space permanent-multipole field at every site, (N, 3)."""
    t = terms if terms is not None else pair_terms(sys, setup)
    b1, b2, b3 = t.permanent_coeffs()
    i, j, r = t.i, t.j, t.r
    e_i = multipole_field(r, sys.q[j], sys.dip[j], sys.quad[j], b1, b2, b3)
    e_j = multipole_field(-r, sys.q[i], sys.dip[i], sys.quad[i], b1, b2, b3)
    return scatter_add(sys.n, i, e_i) + scatter_add(sys.n, j, e_j)


def dipole_field_real(sys, setup, mu, terms: PairTerms | None = None) -> np.ndarray:
    """Real-space part of T*mu at every site; mu (N, 3) or (N, 3, nb)."""
    t = terms if terms is not None else pair_terms(sys, setup)
    b1u, b2u = t.mutual_coeffs()
    i, j, r = t.i, t.j, t.r
    return scatter_add(sys.n, i, dipole_field(r, mu[j], b1u, b2u)) + \
        scatter_add(sys.n, j, dipole_field(-r, mu[i], b1u, b2u))


def _row_terms(sys, setup, a):
    """PairTerms of site a with every other site in range (direct O(N) scan)."""
    others = np.concatenate([np.arange(a), np.arange(a + 1, sys.n)])
    r = minimum_image(sys.xyz[a] - sys.xyz[others], setup.box if setup.periodic else None)
    if setup.periodic:
        r2 = r[:, 0] * r[:, 0] + r[:, 1] * r[:, 1] + r[:, 2] * r[:, 2]
        keep = r2 < setup.cutoff * setup.cutoff
        others, r = others[keep], r[keep]
    ii = np.full(others.shape, a, dtype=np.int64)
    return PairTerms(sys, setup, ii, others, r)


def permanent_field_real_rows(sys, setup, rows) -> np.ndarray:
    """Real-space permanent field at the given sites only, by direct scan."""
    out = np.zeros((len(rows), 3))
    for k, a in enumerate(rows):
        t = _row_terms(sys, setup, int(a))
        b1, b2, b3 = t.permanent_coeffs()
        j = t.j
        out[k] = multipole_field(t.r, sys.q[j], sys.dip[j], sys.quad[j], b1, b2, b3).sum(0)
    return out


def dipole_field_real_rows(sys, setup, mu, rows) -> np.ndarray:
    """Real-space T*mu at the given sites only, by direct scan."""
    out = np.zeros((len(rows), 3))
    for k, a in enumerate(rows):
        t = _row_terms(sys, setup, int(a))
        b1u, b2u = t.mutual_coeffs()
        out[k] = dipole_field(t.r, mu[t.j], b1u, b2u).sum(0)
    return out

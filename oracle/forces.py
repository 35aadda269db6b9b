"""Gradients of the polarization energy (oracle side).

The paper's ``epolar1`` computes the dipole polarization energy and forces
(Section "Hotspots"). At the solution of A mu = E0 the energy
U = C (1/2 mu.A mu - mu.E0) is stationary in mu, so every gradient is taken at
fixed mu (no re-solve):

    F_k   = -dU/dr_k = C [ 1/2 d(mu.T mu)/dr_k + d(mu.E0)/dr_k ]
    dU/dq_k, dU/dd_k, dU/dTheta_k = -C d(mu.E0)/d(moment)

Real space, pair (i, j), r = x_i - x_j:
  mutual   W = mu_i.T_ij mu_j = -B1u (mu_i.mu_j) + B2u (mu_i.r)(mu_j.r)
           dW/dr_i = [-B1u' (mu_i.mu_j) + B2u' (mu_i.r)(mu_j.r)] r/|r|
                     + B2u [mu_i (mu_j.r) + mu_j (mu_i.r)]
  permanent V = mu_i.E_{i<-j}(r) + mu_j.E_{j<-i}(-r), and for a dipole mu in the
           field of a multipole (q, d, Theta) at displacement r:
           grad_r (mu.E) = [B1' (q mu.r - mu.d) + B2' ((d.r)(mu.r) - 2/3 mu.Theta r)
                            + B3' (r.Theta.r)(mu.r)/3] r/|r|
                           + q B1 mu + B2 [d (mu.r) + mu (d.r)] - 2/3 B2 Theta mu
                           + B3/3 [2 Theta r (mu.r) + (r.Theta.r) mu]
  with the damped kernels B_n^eff = B_n - (1 - s l_{2n+1}) bare_n and
  dB_n^eff/dr = -r B_{n+1} + s l' bare_n + (1 - s l) r bare_{n+1},
  l3' = 3x/r e^-x, l5' = 3x^2/r e^-x, l7' = 3x/r (0.6 x^2 - 0.2 x) e^-x.

Reciprocal space (smooth PME): with phi_mu = conv(spread(mu)) and
phi_M = conv(spread(q, d, Theta)), and the interpolated derivatives at atom k,
phi_a = sum_g d_a W_k(g) phi(g) (likewise second and third derivatives),
    F_k,a = -C [ sum_b mu_b (phi_M,ab + phi_mu,ab) + q phi_mu,a
                 + sum_b d_b phi_mu,ab + 1/3 sum_bc Theta_bc phi_mu,abc ]
    dU/dq_k = C phi_mu(k),  dU/dd_k,a = C phi_mu,a(k),
    dU/dTheta_k,ab = C/3 phi_mu,ab(k)  (twice that for the stored off-diagonals)
Self term: dU/dd_k = -C 4 beta^3/(3 sqrt(pi)) mu_k; no force.

Quadrupole gradients are with respect to the six stored numbers
(xx, yy, zz, xy, xz, yz), each off-diagonal standing for two matrix entries.
"""
from __future__ import annotations

import numpy as np

from .ewald import self_field_coefficient
from .pme import PmeGrid
from .realspace import PairTerms, quad_matrix, scatter_add
from .setup import COULOMB

_OFF = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _lambda_derivs(x, dist):
    e = np.exp(-x)
    dxdr = 3.0 * x / dist
    l3p = dxdr * e
    l5p = dxdr * x * e
    l7p = dxdr * (0.6 * x * x - 0.2 * x) * e
    return l3p, l5p, l7p


def _damped(t: PairTerms, n: int, s, lam, lamp):
    """(B_n^eff, dB_n^eff/dr) for scale s and Thole factor lam = l_{2n+1}."""
    r = t.dist
    b = t.B[n] - (1.0 - s * lam) * t.bare[n]
    db = -r * t.B[n + 1] + s * lamp * t.bare[n] + (1.0 - s * lam) * r * t.bare[n + 1]
    return b, db


def _grad_mu_dot_field(r, rhat, mu, q, d, th, b1, b2, b3, db1, db2, db3):
    """grad_r (mu . E(r)) for the field of multipoles (q, d, Theta matrices)."""
    thr = np.einsum("pab,pb->pa", th, r)
    thmu = np.einsum("pab,pb->pa", th, mu)
    rthr = np.einsum("pa,pa->p", r, thr)
    mr = np.einsum("pa,pa->p", mu, r)
    dr = np.einsum("pa,pa->p", d, r)
    md = np.einsum("pa,pa->p", mu, d)
    mthr = np.einsum("pa,pa->p", mu, thr)
    radial = db1 * (q * mr - md) + db2 * (dr * mr - (2.0 / 3.0) * mthr) + db3 * rthr * mr / 3.0
    return (radial[:, None] * rhat + (q * b1)[:, None] * mu
            + b2[:, None] * (d * mr[:, None] + mu * dr[:, None])
            - (2.0 / 3.0) * b2[:, None] * thmu
            + (b3 / 3.0)[:, None] * (2.0 * thr * mr[:, None] + rthr[:, None] * mu))


def _moment_grads(r, mu, b1, b2, b3):
    """d(mu.E)/d(q, d, Theta6) of the source multipole at displacement r."""
    mr = np.einsum("pa,pa->p", mu, r)
    gq = b1 * mr
    gd = -b1[:, None] * mu + (b2 * mr)[:, None] * r
    gt = np.empty((r.shape[0], 6))
    for k, (a, c) in enumerate(_OFF):
        if a == c:
            gt[:, k] = -(2.0 / 3.0) * b2 * mu[:, a] * r[:, a] + b3 * mr * r[:, a] * r[:, a] / 3.0
        else:
            gt[:, k] = (-(2.0 / 3.0) * b2 * (mu[:, a] * r[:, c] + mu[:, c] * r[:, a])
                        + b3 * mr * 2.0 * r[:, a] * r[:, c] / 3.0)
    return gq, gd, gt


def real_space_gradients(sys, setup, mu, t: PairTerms):
    """Real-space (force, dU/dq, dU/dd, dU/dTheta6) at fixed mu."""
    n = sys.n
    i, j, r, dist = t.i, t.j, t.r, t.dist
    rhat = r / dist[:, None]
    l3, l5, l7, _ = t.lam
    l3p, l5p, l7p = _lambda_derivs(t.x, dist)
    one = np.ones_like(dist)
    # mutual (scale 1)
    b1u, db1u = _damped(t, 1, one, l3, l3p)
    b2u, db2u = _damped(t, 2, one, l5, l5p)
    mi, mj = mu[i], mu[j]
    mimj = np.einsum("pa,pa->p", mi, mj)
    mir = np.einsum("pa,pa->p", mi, r)
    mjr = np.einsum("pa,pa->p", mj, r)
    gw = (-db1u * mimj + db2u * mir * mjr)[:, None] * rhat + b2u[:, None] * (mi * mjr[:, None] + mj * mir[:, None])
    # permanent (scale 0 inside a molecule)
    s = t.inter
    b1, db1 = _damped(t, 1, s, l3, l3p)
    b2, db2 = _damped(t, 2, s, l5, l5p)
    b3, db3 = _damped(t, 3, s, l7, l7p)
    thi, thj = quad_matrix(sys.quad[i]), quad_matrix(sys.quad[j])
    g1 = _grad_mu_dot_field(r, rhat, mi, sys.q[j], sys.dip[j], thj, b1, b2, b3, db1, db2, db3)
    g2 = _grad_mu_dot_field(-r, -rhat, mj, sys.q[i], sys.dip[i], thi, b1, b2, b3, db1, db2, db3)
    fpair = COULOMB * (gw + g1 - g2)
    F = scatter_add(n, i, fpair) - scatter_add(n, j, fpair)
    # moment gradients: sources j seen by mu_i at r, sources i seen by mu_j at -r
    gq_j, gd_j, gt_j = _moment_grads(r, mi, b1, b2, b3)
    gq_i, gd_i, gt_i = _moment_grads(-r, mj, b1, b2, b3)
    gq = -COULOMB * (np.bincount(j, gq_j, minlength=n) + np.bincount(i, gq_i, minlength=n))
    gd = -COULOMB * (scatter_add(n, j, gd_j) + scatter_add(n, i, gd_i))
    gt = -COULOMB * (scatter_add(n, j, gt_j) + scatter_add(n, i, gt_i))
    return F, gq, gd, gt


def _gather(g: PmeGrid, phi, dx, dy, dz):
    vals = phi.reshape(-1)[g.flat].reshape(-1, g.n, g.n, g.n)
    return np.einsum("pa,pb,pc,pabc->p", g.wx[dx], g.wy[dy], g.wz[dz], vals)


def recip_gradients(sys, setup, mu, grid: PmeGrid | None = None):
    """Reciprocal-space (force, dU/dq, dU/dd, dU/dTheta6) at fixed mu."""
    g = grid if grid is not None and len(grid.wx) > 3 else PmeGrid(
        sys.xyz, setup.box, setup.grid, setup.order, setup.beta, nderiv=3)
    phi_mu = g.convolve(g.spread_dipoles(mu))
    phi_m = g.convolve(g.spread_multipoles(sys.q, sys.dip, sys.quad))
    e = np.eye(3, dtype=int)
    d1 = {a: tuple(e[a]) for a in range(3)}

    def deriv(phi, *axes):
        o = np.zeros(3, dtype=int)
        for a in axes:
            o[a] += 1
        return _gather(g, phi, o[0], o[1], o[2])

    n = sys.n
    pmu1 = np.stack([deriv(phi_mu, a) for a in range(3)], 1)
    pmu2 = np.empty((n, 3, 3))
    pm2 = np.empty((n, 3, 3))
    for a in range(3):
        for b in range(3):
            pmu2[:, a, b] = deriv(phi_mu, a, b)
            pm2[:, a, b] = deriv(phi_m, a, b)
    pmu3 = np.empty((n, 3, 3, 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                pmu3[:, a, b, c] = deriv(phi_mu, a, b, c)
    th = quad_matrix(sys.quad)
    F = -COULOMB * (np.einsum("pb,pab->pa", mu, pm2 + pmu2) + sys.q[:, None] * pmu1
                    + np.einsum("pb,pab->pa", sys.dip, pmu2)
                    + np.einsum("pbc,pabc->pa", th, pmu3) / 3.0)
    gq = COULOMB * deriv(phi_mu)
    gd = COULOMB * pmu1
    gt = np.empty((n, 6))
    for k, (a, b) in enumerate(_OFF):
        gt[:, k] = COULOMB * pmu2[:, a, b] / 3.0 * (1.0 if a == b else 2.0)
    del d1
    return F, gq, gd, gt


def polarization_gradients(op, mu):
    """(F, dU/dq, dU/dd, dU/dTheta6) of U = -1/2 C mu.E0 at the solution mu."""
    sys, setup = op.sys, op.setup
    F, gq, gd, gt = real_space_gradients(sys, setup, mu, op.terms)
    if setup.periodic:
        Fr, gqr, gdr, gtr = recip_gradients(sys, setup, mu)
        F, gq, gd, gt = F + Fr, gq + gqr, gd + gdr, gt + gtr
        gd = gd - COULOMB * self_field_coefficient(setup.beta) * mu
    return F, gq, gd, gt

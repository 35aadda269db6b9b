"""Truncated conjugate gradient of order one (TCG-1) and its gradients (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's outlook (Section "Perspectives on Tinker-HP 1.2 performance")
names the non-iterative TCG-1 solver of Aviat et al. (JCTC 2017) for the
short-range polarization. Reading used here: one step of the diagonal-
preconditioned conjugate gradient of ``solver`` from the direct guess, with
the energy of that iterate,

    u = alpha E,  r = T u (the residual E - A u),  z = alpha r,
    gamma = (r.z) / (z.A z),  mu_1 = u + gamma z,  U_1 = -1/2 C mu_1 . E,

and, since mu_1 is not the minimiser, gradients that differentiate through
gamma, r and z (no stationarity shortcut). With w = u.T u, s = r.z,
t = z.A z = s - z.T z, v = alpha T z, and dT, dE the derivatives of the
operator and of the permanent field:

    dU_1 = -1/2 C [ c.dE + (w/t)(2(1-gamma) z.dT u + 2 gamma v.dT u + gamma z.dT z)
                    + gamma u.dT u ],
    c = 2 u + (w/t)(2(1-gamma) v + 2 gamma alpha T v) + 2 gamma z,

from d(u.E) = 2 u.dE, dw = 2 z.dE + u.dT u, d s = 2 z.dT u + 2 v.dE,
d(z.T z) = 2 v.dT u + 2 (alpha T v).dE + z.dT z and
d gamma = ((1-gamma) ds + gamma d(z.T z)) / t. The multipoles enter only
through E, so the moment gradients are those of -1/2 C c.E at fixed c.

Building blocks (each pinned by finite differences in the tests):
  field_gradients(c):        d(c.E)/dx and d(c.E)/d(q, d, Theta) at fixed c
  bilinear_T_gradient(a, b): d(a.T b)/dx at fixed a, b
"""
from __future__ import annotations

import numpy as np

from .ewald import self_field_coefficient
from .forces import _OFF, _damped, _grad_mu_dot_field, _lambda_derivs, _moment_grads
from .pme import PmeGrid
from .realspace import quad_matrix, scatter_add
from .setup import COULOMB


def _grid3(sys, setup):
    return PmeGrid(sys.xyz, setup.box, setup.grid, setup.order, setup.beta, nderiv=3)


def _deriv(g: PmeGrid, phi, *axes):
    o = [0, 0, 0]
    for a in axes:
        o[a] += 1
    vals = phi.reshape(-1)[g.flat].reshape(-1, g.n, g.n, g.n)
    return np.einsum("pa,pb,pc,pabc->p", g.wx[o[0]], g.wy[o[1]], g.wz[o[2]], vals)


def _hessians(g, phi, n):
    h = np.empty((n, 3, 3))
    for a in range(3):
        for b in range(3):
            h[:, a, b] = _deriv(g, phi, a, b)
    return h


def field_gradients(op, c, scale=None):
    """(d(c.E)/dx (N,3), d/dq (N,), d/dd (N,3), d/dTheta6 (N,6)) at fixed c.

    scale: per-pair scale of the permanent field (default: 0 inside a
    molecule, 1 otherwise)."""
    sys, setup, t = op.sys, op.setup, op.terms
    n = sys.n
    i, j, r, dist = t.i, t.j, t.r, t.dist
    rhat = r / dist[:, None]
    l3, l5, l7, _ = t.lam
    l3p, l5p, l7p = _lambda_derivs(t.x, dist)
    s = t.inter if scale is None else scale
    b1, db1 = _damped(t, 1, s, l3, l3p)
    b2, db2 = _damped(t, 2, s, l5, l5p)
    b3, db3 = _damped(t, 3, s, l7, l7p)
    thi, thj = quad_matrix(sys.quad[i]), quad_matrix(sys.quad[j])
    ci, cj = c[i], c[j]
    g1 = _grad_mu_dot_field(r, rhat, ci, sys.q[j], sys.dip[j], thj, b1, b2, b3, db1, db2, db3)
    g2 = _grad_mu_dot_field(-r, -rhat, cj, sys.q[i], sys.dip[i], thi, b1, b2, b3, db1, db2, db3)
    gx = scatter_add(n, i, g1 - g2) - scatter_add(n, j, g1 - g2)
    gq_j, gd_j, gt_j = _moment_grads(r, ci, b1, b2, b3)
    gq_i, gd_i, gt_i = _moment_grads(-r, cj, b1, b2, b3)
    gq = np.bincount(j, gq_j, minlength=n) + np.bincount(i, gq_i, minlength=n)
    gd = scatter_add(n, j, gd_j) + scatter_add(n, i, gd_i)
    gt = scatter_add(n, j, gt_j) + scatter_add(n, i, gt_i)
    if setup.periodic:
        g = _grid3(sys, setup)
        phi_m = g.convolve(g.spread_multipoles(sys.q, sys.dip, sys.quad))
        phi_c = g.convolve(g.spread_dipoles(c))
        hm, hc = _hessians(g, phi_m, n), _hessians(g, phi_c, n)
        pc1 = np.stack([_deriv(g, phi_c, a) for a in range(3)], 1)
        pc3 = np.empty((n, 3, 3, 3))
        for a in range(3):
            for b in range(3):
                for e in range(3):
                    pc3[:, a, b, e] = _deriv(g, phi_c, a, b, e)
        th = quad_matrix(sys.quad)
        # c.E_rec = -<phi_c, Q_M>: both the field points and the sources move
        gx = gx - (np.einsum("pb,pab->pa", c, hm) + sys.q[:, None] * pc1
                   + np.einsum("pb,pab->pa", sys.dip, hc) + np.einsum("pbc,pabc->pa", th, pc3) / 3.0)
        gq = gq - _deriv(g, phi_c)
        gd = gd - pc1
        for k, (a, b) in enumerate(_OFF):
            gt[:, k] -= hc[:, a, b] / 3.0 * (1.0 if a == b else 2.0)
        gd = gd + self_field_coefficient(setup.beta) * c
    return gx, gq, gd, gt


def bilinear_T_gradient(op, a, b):
    """d(a.T b)/dx (N, 3) at fixed a, b (T = real + reciprocal + self)."""
    sys, setup, t = op.sys, op.setup, op.terms
    n = sys.n
    i, j, r, dist = t.i, t.j, t.r, t.dist
    rhat = r / dist[:, None]
    l3, l5, _, _ = t.lam
    l3p, l5p, _ = _lambda_derivs(t.x, dist)
    one = np.ones_like(dist)
    b1u, db1u = _damped(t, 1, one, l3, l3p)
    b2u, db2u = _damped(t, 2, one, l5, l5p)

    def grad_w(x, y):  # grad_r of x.T(r) y = -B1u x.y + B2u (x.r)(y.r)
        xy = np.einsum("pa,pa->p", x, y)
        xr = np.einsum("pa,pa->p", x, r)
        yr = np.einsum("pa,pa->p", y, r)
        return (-db1u * xy + db2u * xr * yr)[:, None] * rhat + b2u[:, None] * (x * yr[:, None] + y * xr[:, None])

    gp = grad_w(a[i], b[j]) + grad_w(a[j], b[i])
    gx = scatter_add(n, i, gp) - scatter_add(n, j, gp)
    if setup.periodic:
        g = _grid3(sys, setup)
        ha = _hessians(g, g.convolve(g.spread_dipoles(a)), n)
        hb = _hessians(g, g.convolve(g.spread_dipoles(b)), n)
        # a.T_rec b = -<S_a, G * S_b>: each spread moves with its atom
        gx = gx - (np.einsum("pb,pab->pa", a, hb) + np.einsum("pb,pab->pa", b, ha))
    return gx


def tcg1(op):
    """(U_1 kcal/mol, mu_1, intermediates) of one preconditioned CG step from alpha E."""
    sys = op.sys
    al = sys.alpha[:, None]
    E = op.permanent_field()
    u = al * E
    r = op.apply_T(u)
    z = al * r
    y = op.apply_T(z)
    v = al * y
    s = float((r * z).sum())
    t = s - float((z * y).sum())
    gamma = s / t
    mu1 = u + gamma * z
    U = -0.5 * COULOMB * float((mu1 * E).sum())
    return U, mu1, dict(E=E, u=u, r=r, z=z, v=v, s=s, t=t, gamma=gamma, w=float((u * r).sum()))


def tcg1_gradients(op):
    """(F = -dU_1/dx, dU_1/dq, dU_1/dd, dU_1/dTheta6) of the TCG-1 energy."""
    _, _, k = tcg1(op)
    al = op.sys.alpha[:, None]
    u, z, v, w, t, gm = k["u"], k["z"], k["v"], k["w"], k["t"], k["gamma"]
    Tv = op.apply_T(v)
    c = 2.0 * u + (w / t) * (2.0 * (1.0 - gm) * v + 2.0 * gm * al * Tv) + 2.0 * gm * z
    gx, gq, gd, gt = field_gradients(op, c)
    bil = ((w / t) * (2.0 * (1.0 - gm) * bilinear_T_gradient(op, z, u) + 2.0 * gm * bilinear_T_gradient(op, v, u)
                      + gm * bilinear_T_gradient(op, z, z)) + gm * bilinear_T_gradient(op, u, u))
    h = -0.5 * COULOMB
    return -h * (gx + bil), h * gq, h * gd, h * gt

"""Two right-hand sides: direct- and polarization-scaled permanent fields (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

General AMOEBA computes the permanent field twice, with two exclusion rules
for nearby pairs (paper, Section "Polarizable AMOEBA force field" names the
model; the scaling rules are Ren & Ponder's): a "direct" field E_d and a
"polarization" field E_p, and solves for one dipole set per field with the
same operator A. Here the two rules differ only inside a molecule: E_d uses
scale 0 (the rule of ``realspace``) and E_p a scale s_p in [0, 1], i.e. the
damped kernel B_n - (1 - s lambda_{2n+1}) bare_n with s = s_p for two sites of
one molecule and 1 otherwise. With mu_d = A^-1 E_d and mu_p = A^-1 E_p,

    U = -1/2 C mu_d . E_p  (= -1/2 C mu_p . E_d, A being symmetric),

and since d(A^-1) = A^-1 dT A^-1,

    dU = -1/2 C [ mu_p . dE_d + mu_d . dE_p + mu_p . dT mu_d ].

With s_p = 0 both fields coincide and U is the one-field energy of ``energy``.
"""
from __future__ import annotations

import numpy as np

from .ewald import self_field_coefficient
from .pme import PmeGrid, permanent_field_recip
from .realspace import multipole_field, scatter_add
from .setup import COULOMB
from .solver import solve
from .tcg import bilinear_T_gradient, field_gradients


def pair_scale(op, s_intra: float) -> np.ndarray:
    """Per-pair scale: 1 between molecules, s_intra inside one."""
    inter = op.terms.inter
    return inter + (1.0 - inter) * s_intra


def permanent_field_scaled(op, s_intra: float) -> np.ndarray:
    """Permanent field with scale s_intra for the pairs inside a molecule."""
    sys, setup, t = op.sys, op.setup, op.terms
    s = pair_scale(op, s_intra)
    l3, l5, l7, _ = t.lam
    b1 = t.B[1] - (1.0 - s * l3) * t.bare[1]
    b2 = t.B[2] - (1.0 - s * l5) * t.bare[2]
    b3 = t.B[3] - (1.0 - s * l7) * t.bare[3]
    i, j, r = t.i, t.j, t.r
    e = scatter_add(sys.n, i, multipole_field(r, sys.q[j], sys.dip[j], sys.quad[j], b1, b2, b3)) + \
        scatter_add(sys.n, j, multipole_field(-r, sys.q[i], sys.dip[i], sys.quad[i], b1, b2, b3))
    if setup.periodic:
        g = op.grid if op.grid is not None else PmeGrid(sys.xyz, setup.box, setup.grid, setup.order, setup.beta)
        e = e + permanent_field_recip(sys, setup, g) + self_field_coefficient(setup.beta) * sys.dip
    return e


def two_rhs_solve(op, s_p: float, tol: float = 1e-12, max_iter: int = 500):
    """(U kcal/mol, mu_d, mu_p, E_d, E_p)."""
    e_d = permanent_field_scaled(op, 0.0)
    e_p = permanent_field_scaled(op, s_p)
    mu_d, _, _ = solve(op, e_d, tol, max_iter)
    mu_p, _, _ = solve(op, e_p, tol, max_iter)
    U = -0.5 * COULOMB * float((mu_d * e_p).sum())
    return U, mu_d, mu_p, e_d, e_p


def two_rhs_gradients(op, s_p: float, mu_d, mu_p):
    """(F = -dU/dx, dU/dq, dU/dd, dU/dTheta6) at the two solutions."""
    gd_x, gd_q, gd_d, gd_t = field_gradients(op, mu_p, scale=pair_scale(op, 0.0))
    gp_x, gp_q, gp_d, gp_t = field_gradients(op, mu_d, scale=pair_scale(op, s_p))
    bil = bilinear_T_gradient(op, mu_p, mu_d)
    h = -0.5 * COULOMB
    return -h * (gd_x + gp_x + bil), h * (gd_q + gp_q), h * (gd_d + gp_d), h * (gd_t + gp_t)


"""Screened Coulomb kernels and Thole damping (oracle side).

The paper gives no formulas; AMOEBA's damped point-dipole model is the one it
names in Section "Polarizable AMOEBA force field" (Ren & Ponder 2003, Thole
1981) and the real-space Ewald kernels are the standard multipolar ones
(Smith 1998; Sagui, Pedersen & Darden 2004).

B_n(r): for field point minus source r, |r| = r,
    B_0 = erfc(beta r) / r
    B_n = [ (2n-1) B_{n-1} + (2 beta^2)^n / (beta sqrt(pi)) exp(-beta^2 r^2) ] / r^2
With beta = 0 they reduce to the bare 1/r, 1/r^3, 3/r^5, 15/r^7, 105/r^9.

Thole (AMOEBA exponential form): x = a r^3 / sqrt(alpha_i alpha_j),
a = min(a_i, a_j),
    lambda_3 = 1 - e^-x
    lambda_5 = 1 - (1 + x) e^-x
    lambda_7 = 1 - (1 + x + 0.6 x^2) e^-x
    lambda_9 = 1 - (1 + x + (18/35) x^2 + (9/35) x^3) e^-x
The damped coefficient of order n is B_n - (1 - s lambda_{2n+1}) bare_n with
s the pair scale (0 for excluded pairs, 1 otherwise).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

SQRT_PI = float(np.sqrt(np.pi))


def screened_B(r: np.ndarray, beta: float, nmax: int) -> list[np.ndarray]:
    """[B_0, ..., B_nmax] at distances r (array), Ewald-screened if beta > 0."""
    r = np.asarray(r, dtype=np.float64)
    r2 = r * r
    out = []
    if beta > 0.0:
        b = erfc(beta * r) / r
        out.append(b)
        ex = np.exp(-beta * beta * r2)
        fac = ex / (beta * SQRT_PI)
        for n in range(1, nmax + 1):
            fac = fac * (2.0 * beta * beta)
            b = ((2 * n - 1) * b + fac) / r2
            out.append(b)
    else:
        b = 1.0 / r
        out.append(b)
        for n in range(1, nmax + 1):
            b = (2 * n - 1) * b / r2
            out.append(b)
    return out


def thole_x(r, alpha_i, alpha_j, a_i, a_j):
    """Thole argument x = min(a_i, a_j) r^3 / sqrt(alpha_i alpha_j)."""
    a = np.minimum(a_i, a_j)
    return a * r ** 3 / np.sqrt(alpha_i * alpha_j)


def thole_lambdas(x: np.ndarray):
    """(lambda_3, lambda_5, lambda_7, lambda_9) for Thole argument x."""
    e = np.exp(-x)
    l3 = 1.0 - e
    l5 = 1.0 - (1.0 + x) * e
    l7 = 1.0 - (1.0 + x + 0.6 * x * x) * e
    l9 = 1.0 - (1.0 + x + (18.0 / 35.0) * x * x + (9.0 / 35.0) * x ** 3) * e
    return l3, l5, l7, l9


def self_field_coefficient(beta: float) -> float:
    """Ewald self field per unit dipole, 4 beta^3 / (3 sqrt(pi))."""
    return 4.0 * beta ** 3 / (3.0 * SQRT_PI)

"""Polarization energy (oracle side).

At the solution of A mu = E0 the polarization energy (paper, Section
"Hotspots": ``epolar1`` computes the dipole polarization energy and forces) is

    U = -1/2 C sum_i mu_i . E0_i          (kcal/mol),

which equals C (1/2 mu.A mu - mu.E0), the minimum of the quadratic form over
mu (the value the pins check).
"""
from __future__ import annotations

import numpy as np

from .setup import COULOMB


def polarization_energy(mu: np.ndarray, E0: np.ndarray) -> float:
    return float(-0.5 * COULOMB * (mu * E0).sum())


def quadratic_form_energy(apply_A, mu: np.ndarray, E0: np.ndarray) -> float:
    """C (1/2 mu.A mu - mu.E0): equals the energy above at the exact solution."""
    return float(COULOMB * (0.5 * (mu * apply_A(mu)).sum() - (mu * E0).sum()))

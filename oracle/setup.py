"""Settings of one electrostatics evaluation (oracle side).

Units: Angstrom, elementary charge e, field in e/Angstrom^2, energy in
kcal/mol through COULOMB. Debye per e*Angstrom is DEBYE.
"""
from __future__ import annotations

from dataclasses import dataclass

COULOMB = 332.0637133      # kcal*Angstrom/(mol*e^2)
DEBYE = 4.8032047          # Debye per e*Angstrom


@dataclass(frozen=True)
class Setup:
    """Ewald / PME settings.

    box     cubic box edge (Angstrom) or None for an isolated cluster
            (then: no cutoff, beta = 0, no reciprocal or self terms)
    cutoff  real-space cutoff, must be < box/2 (minimum image)
    beta    Ewald splitting parameter (1/Angstrom)
    grid    PME grid points per axis
    order   B-spline order (5: piecewise quartic, 5 points per axis)
    """

    box: float | None
    cutoff: float = 7.0
    beta: float = 0.5446
    grid: int = 24
    order: int = 5

    @property
    def periodic(self) -> bool:
        return self.box is not None

    @staticmethod
    def cluster() -> "Setup":
        return Setup(box=None, cutoff=float("inf"), beta=0.0, grid=0, order=5)

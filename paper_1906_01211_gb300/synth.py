"""Seeded synthetic AMOEBA-like water systems.

This module only draws inputs: positions, permanent multipoles and
polarization parameters. It holds none of the polarization arithmetic, so the
CUDA path and the CPU oracle can both be fed from it without sharing any of
the method.

The paper's benchmark systems (the DHFR protein in water and the 96,000-atom
"Puddle" water box, listed in its table of test systems in Section
"Execution setup") and the AMOEBA parameter files are not available, so the
workloads are seeded stand-ins of the same sizes. AMOEBA itself (distributed
multipoles through quadrupoles, Thole-damped point-dipole polarization) is
named in Section "Polarizable AMOEBA force field"; the numbers below are
synthetic, AMOEBA-water-like values.

Recipe (fixed order of draws from ``numpy.random.Generator(PCG64(seed))``):

1. ``m = ceil(n ** (1/3))`` lattice sites per axis, spacing ``s = L / m``,
   site centres ``(i + 1/2) s``. If ``m**3 > n``, ``n`` sites are chosen as the
   first ``n`` entries of a seeded permutation, then put back in lattice order.
2. Oxygen jitter: ``U(-0.3, 0.3)`` Angstrom per component.
3. Orientation: a uniformly random rotation from a normalised 4-vector of
   standard normals (a unit quaternion).
4. Permanent dipoles: ``N(0, 0.05)`` e*Angstrom per component (sigma = 0.05).
5. Quadrupoles: six components ``xx, yy, zz, xy, xz, yz`` drawn ``N(0, 0.1)``
   e*Angstrom^2, then trace/3 subtracted from the diagonal (traceless).

Atoms are ordered O, H, H per water; ``mol`` is the water index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OH_BOND = 0.9572          # Angstrom
HOH_ANGLE_DEG = 104.52
Q_O, Q_H = -0.51966, 0.25983
ALPHA_O, ALPHA_H = 0.837, 0.496   # Angstrom^3
THOLE_A = 0.39
WATER_DENSITY = 0.0334    # waters per Angstrom^3


@dataclass
class System:
    """A set of polarizable sites, all arrays float64 unless noted.

    xyz   (N, 3) positions, Angstrom (periodic boxes: not wrapped)
    q     (N,)   charges, e
    dip   (N, 3) permanent dipoles, global frame, e*Angstrom
    quad  (N, 6) traceless quadrupoles xx, yy, zz, xy, xz, yz, e*Angstrom^2
    alpha (N,)   polarizabilities, Angstrom^3
    thole (N,)   Thole damping parameters (dimensionless)
    mol   (N,)   int32 molecule index; pairs within a molecule are excluded
                 from the permanent field
    box   cubic box edge in Angstrom, or None for an isolated cluster
    """

    xyz: np.ndarray
    q: np.ndarray
    dip: np.ndarray
    quad: np.ndarray
    alpha: np.ndarray
    thole: np.ndarray
    mol: np.ndarray
    box: float | None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def _body_frame_water() -> np.ndarray:
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
        [-OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
    ])


def _quat_to_matrix(qt: np.ndarray) -> np.ndarray:
    w, x, y, z = qt[:, 0], qt[:, 1], qt[:, 2], qt[:, 3]
    R = np.empty((qt.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def make_waters(n_waters: int, L: float, seed: int, periodic: bool = True) -> System:
    """Water system on a jittered lattice in a cube of edge ``L`` (see module doc)."""
    if n_waters < 1:
        raise ValueError("n_waters must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 1
    while m ** 3 < n_waters:
        m += 1
    s = L / m
    idx = np.arange(m ** 3)
    if m ** 3 > n_waters:
        idx = np.sort(rng.permutation(m ** 3)[:n_waters])
    ix, iy, iz = idx // (m * m), (idx // m) % m, idx % m
    sites = (np.stack([ix, iy, iz], axis=1) + 0.5) * s
    sites = sites + rng.uniform(-0.3, 0.3, size=(n_waters, 3))
    quat = rng.standard_normal((n_waters, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    R = _quat_to_matrix(quat)
    body = _body_frame_water()
    xyz = sites[:, None, :] + np.einsum("wab,kb->wka", R, body)
    xyz = xyz.reshape(-1, 3)
    n = 3 * n_waters
    dip = rng.normal(0.0, 0.05, size=(n, 3))
    quad = rng.normal(0.0, 0.1, size=(n, 6))
    tr = (quad[:, 0] + quad[:, 1] + quad[:, 2]) / 3.0
    quad[:, 0] -= tr
    quad[:, 1] -= tr
    quad[:, 2] -= tr
    q = np.tile([Q_O, Q_H, Q_H], n_waters).astype(np.float64)
    alpha = np.tile([ALPHA_O, ALPHA_H, ALPHA_H], n_waters).astype(np.float64)
    thole = np.full(n, THOLE_A)
    mol = np.repeat(np.arange(n_waters, dtype=np.int32), 3)
    return System(xyz=np.ascontiguousarray(xyz), q=q, dip=dip, quad=quad,
                  alpha=alpha, thole=thole, mol=mol,
                  box=float(L) if periodic else None,
                  meta={"n_waters": n_waters, "seed": seed, "L": float(L)})


def water_frames(n_waters: int):
    """Local-frame topology of the waters of ``make_waters`` (O, H, H order):
    (kind, z atom, x atom) per site, AMOEBA's water convention. Oxygen:
    bisector (kind 1) of its two hydrogens; each hydrogen: Z-then-X (kind 0)
    with z toward its oxygen and x toward the other hydrogen. With these
    frames the drawn dipoles and quadrupoles are read as local-frame values.
    Topology only: the frames themselves are computed by the method."""
    base = 3 * np.arange(n_waters, dtype=np.int32)
    kind = np.tile(np.array([1, 0, 0], dtype=np.int32), n_waters)
    zatom = np.stack([base + 1, base, base], axis=1).reshape(-1)
    xatom = np.stack([base + 2, base + 2, base + 1], axis=1).reshape(-1)
    return kind, zatom.astype(np.int32), xatom.astype(np.int32)


def density_box_edge(n_waters: int) -> float:
    """Edge of a cube holding ``n_waters`` at 0.0334 waters per Angstrom^3."""
    return (n_waters / WATER_DENSITY) ** (1.0 / 3.0)


@dataclass(frozen=True)
class Workload:
    """A named workload: system size, Ewald/PME settings and solver tolerance."""

    name: str
    n_waters: int
    L: float
    grid: int
    tol_debye: float
    precision: str
    seed: int
    cutoff: float = 7.0
    beta: float = 0.5446
    order: int = 5

    def system(self) -> System:
        return make_waters(self.n_waters, self.L, self.seed, periodic=True)


# Workloads shaped like the paper's benchmark systems (table of test systems,
# Section "Execution setup"): 648 atoms (small check case), 23,556 atoms
# (DHFR-sized) and 96,000 atoms (the size of the "Puddle" water box).
WATER_648 = Workload("water-648", 216, 18.643, 24, 1e-8, "fp64", 0)
WATER_23556 = Workload("water-23556", 7852, 62.23, 64, 1e-5, "fp64", 1)
WATER_96000 = Workload("water-96000", 32000, 98.65, 100, 1e-5, "mixed", 2)
WORKLOADS = {w.name: w for w in (WATER_648, WATER_23556, WATER_96000)}


def small_box_settings(L: float, cutoff: float = 7.0):
    """Cutoff, Ewald beta and PME grid for a small periodic box.

    The cutoff is capped below L/2, beta keeps erfc(beta*rc) at the value of
    the 7 Angstrom / 0.5446 setting, and the grid is the smallest 2,3,5-smooth
    size >= L*beta/0.5446 (at least 8).
    """
    rc = min(cutoff, L / 2.0 - 1e-6)
    beta = 3.8122 / rc
    need = max(8, int(math.ceil(L * beta / 0.5446)))
    k = need
    while True:
        v = k
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        if v == 1:
            break
        k += 1
    return rc, beta, k

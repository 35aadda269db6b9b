"""Pair enumeration (oracle side).

The paper's compute routines loop over the atoms, select neighbours by a
cutoff and then loop over the selected sites (Section "General Structure");
its cell-based list builder is ``mlistcell`` (Section "Hotspots"). The oracle
does not mimic a cell list: it takes every unordered pair whose minimum-image
distance is below the cutoff, found with scipy's periodic k-d tree (a library
search primitive) and then re-decided exactly in float64 by the plain rule

    d = x_i - x_j;  d -= L * rint(d / L);  keep if d.d < rc^2.

``brute_force_pairs`` is the O(N^2) definition, used to pin the fast one.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def minimum_image(d: np.ndarray, L: float | None) -> np.ndarray:
    """Wrap displacement vectors into the nearest periodic image."""
    if L is None:
        return d
    return d - L * np.rint(d / L)


def _wrap(xyz: np.ndarray, L: float) -> np.ndarray:
    w = xyz - L * np.floor(xyz / L)
    w[w >= L] -= L
    w[w < 0] += L
    w[w >= L] = 0.0
    return w


def periodic_pairs(xyz: np.ndarray, L: float, rc: float):
    """Unordered pairs (i < j) with minimum-image distance < rc (rc < L/2).

    Returns (i, j, r) with r = minimum_image(x_i - x_j), shape (P, 3).
    """
    if not rc < 0.5 * L:
        raise ValueError("cutoff must be below half the box edge")
    tree = cKDTree(_wrap(xyz, L), boxsize=L)
    cand = tree.query_pairs(rc * (1.0 + 1e-9) + 1e-9, output_type="ndarray")
    if cand.size == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros((0, 3))
    i = np.minimum(cand[:, 0], cand[:, 1]).astype(np.int64)
    j = np.maximum(cand[:, 0], cand[:, 1]).astype(np.int64)
    r = minimum_image(xyz[i] - xyz[j], L)
    r2 = r[:, 0] * r[:, 0] + r[:, 1] * r[:, 1] + r[:, 2] * r[:, 2]
    keep = r2 < rc * rc
    i, j, r = i[keep], j[keep], r[keep]
    order = np.lexsort((j, i))
    return i[order], j[order], r[order]


def cluster_pairs(xyz: np.ndarray):
    """All unordered pairs (i < j) of an isolated cluster, r = x_i - x_j."""
    n = xyz.shape[0]
    i, j = np.triu_indices(n, k=1)
    return i.astype(np.int64), j.astype(np.int64), xyz[i] - xyz[j]


def brute_force_pairs(xyz: np.ndarray, L: float, rc: float):
    """O(N^2) double loop over i < j with the minimum-image rule (small N only)."""
    n = xyz.shape[0]
    out_i, out_j = [], []
    for a in range(n):
        d = minimum_image(xyz[a] - xyz[a + 1:], L)
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        js = np.nonzero(r2 < rc * rc)[0] + a + 1
        out_i.extend([a] * len(js))
        out_j.extend(js.tolist())
    return np.array(out_i, dtype=np.int64), np.array(out_j, dtype=np.int64)


def pairs_for(xyz: np.ndarray, setup):
    """Pairs for a Setup: periodic within the cutoff, or all pairs of a cluster."""
    if setup.periodic:
        return periodic_pairs(xyz, setup.box, setup.cutoff)
    return cluster_pairs(xyz)

"""Local-frame multipoles and the forces from their frames (oracle side).

TEST INFRASTRUCTURE ONLY (see the package header).

AMOEBA (named in the paper's Section "Polarizable AMOEBA force field"; the
frame conventions are Ren & Ponder's) gives each site's dipole and quadrupole
in a local frame fixed by neighbouring atoms, so the global moments turn with
the molecule. For site i with axis atoms zi and xi, v1 = x_zi - x_i,
v2 = x_xi - x_i:

  Z-then-X  (kind 0): e_z = v1/|v1|
  bisector  (kind 1): e_z = a/|a|, a = v1/|v1| + v2/|v2|
  then for both: b = v2 - (v2.e_z) e_z, e_x = b/|b|, e_y = e_z x e_x;
  R = [e_x e_y e_z] (columns), d = R d_loc, Theta = R Theta_loc R^T.

Charges are frame-free. A site with kind -1 keeps its moments as given
(global). With moments tied to the frames, every energy U(x, M(x)) gains
frame terms in its forces:

  F_k = -dU/dx_k|_M - sum_i [ dU/dd_i . dd_i/dx_k + sum_6 dU/dTheta6_i dTheta6_i/dx_k ],
  dd_i/dx = dR d_loc,  dTheta_i/dx = dR Theta_loc R^T + R Theta_loc dR^T,

with dU/dM the moment gradients of the energy at fixed frames and the frame
derivatives from d(v/|v|) = (I - e e^T) dv / |v| and the product rule.
"""
from __future__ import annotations

import numpy as np

from .realspace import quad_matrix


def _unit(v):
    n = np.linalg.norm(v, axis=-1, keepdims=True)
    return v / n, n


def _dunit(e, n, dv):
    """d(v/|v|) for dv (N, 3): (dv - e (e.dv)) / |v|."""
    return (dv - e * np.einsum("pa,pa->p", e, dv)[:, None]) / n


def frames(xyz, kind, zatom, xatom):
    """R (N, 3, 3) with columns e_x, e_y, e_z (identity where kind < 0)."""
    R = np.tile(np.eye(3), (xyz.shape[0], 1, 1))
    m = kind >= 0
    if not m.any():
        return R
    idx = np.nonzero(m)[0]
    ez, ex, ey = _axes(xyz, kind[idx], idx, zatom[idx], xatom[idx])
    R[idx] = np.stack([ex, ey, ez], axis=2)
    return R


def _axes(xyz, kind, i, zi, xi):
    v1, v2 = xyz[zi] - xyz[i], xyz[xi] - xyz[i]
    u1, _ = _unit(v1)
    u2, _ = _unit(v2)
    a = np.where((kind == 1)[:, None], u1 + u2, v1)
    ez, _ = _unit(a)
    b = v2 - ez * np.einsum("pa,pa->p", v2, ez)[:, None]
    ex, _ = _unit(b)
    return ez, ex, np.cross(ez, ex)


def frame_jacobian(xyz, kind, zatom, xatom):
    """dR/dx for every framed site: dict (site i) -> list of (atom k, (3, 3, 3) array
    J[c] = dR/dx_{k,c}) over the site itself, its z atom and its x atom."""
    out = {}
    for i in np.nonzero(kind >= 0)[0]:
        zi, xi = int(zatom[i]), int(xatom[i])
        v1, v2 = xyz[zi] - xyz[i], xyz[xi] - xyz[i]
        n1, n2 = np.linalg.norm(v1), np.linalg.norm(v2)
        u1, u2 = v1 / n1, v2 / n2
        a = u1 + u2 if kind[i] == 1 else v1
        na = np.linalg.norm(a)
        ez = a / na
        b = v2 - (v2 @ ez) * ez
        nb = np.linalg.norm(b)
        ex = b / nb
        jac = []
        for k, s1, s2 in ((int(i), -1.0, -1.0), (zi, 1.0, 0.0), (xi, 0.0, 1.0)):
            J = np.zeros((3, 3, 3))
            for c in range(3):
                dv1, dv2 = np.zeros(3), np.zeros(3)
                dv1[c], dv2[c] = s1, s2
                if kind[i] == 1:
                    da = (dv1 - u1 * (u1 @ dv1)) / n1 + (dv2 - u2 * (u2 @ dv2)) / n2
                else:
                    da = dv1
                dez = (da - ez * (ez @ da)) / na
                db = dv2 - (dv2 @ ez) * ez - (v2 @ dez) * ez - (v2 @ ez) * dez
                dex = (db - ex * (ex @ db)) / nb
                dey = np.cross(dez, ex) + np.cross(ez, dex)
                J[c] = np.stack([dex, dey, dez], axis=1)
            jac.append((k, J))
        # the same atom may appear twice (not in valid frames); merge by atom
        merged = {}
        for k, J in jac:
            merged[k] = merged.get(k, 0.0) + J
        out[int(i)] = list(merged.items())
    return out


def _store6(th):
    return np.stack([th[..., 0, 0], th[..., 1, 1], th[..., 2, 2], th[..., 0, 1], th[..., 0, 2], th[..., 1, 2]], -1)


def global_moments(xyz, dip_loc, quad_loc, kind, zatom, xatom):
    """(d (N, 3), Theta6 (N, 6)) in the global frame."""
    R = frames(xyz, kind, zatom, xatom)
    d = np.einsum("pab,pb->pa", R, dip_loc)
    th = np.einsum("pab,pbc,pdc->pad", R, quad_matrix(quad_loc), R)
    return d, _store6(th)


def frame_forces(xyz, dip_loc, quad_loc, kind, zatom, xatom, gd, gt):
    """Extra forces -sum_i dU/dM_i . dM_i/dx_k (N, 3), from the moment gradients
    gd (N, 3) and gt (N, 6, stored numbers) of an energy at fixed frames."""
    R = frames(xyz, kind, zatom, xatom)
    jac = frame_jacobian(xyz, kind, zatom, xatom)
    th_loc = quad_matrix(quad_loc)
    F = np.zeros_like(xyz)
    for i, parts in jac.items():
        for k, J in parts:
            for c in range(3):
                dR = J[c]
                dd = dR @ dip_loc[i]
                dth = dR @ th_loc[i] @ R[i].T + R[i] @ th_loc[i] @ dR.T
                F[k, c] -= gd[i] @ dd + gt[i] @ _store6(dth)
    return F

"""Error measures of the parity tests (GPU result a against oracle b, both
[N][3] per-atom vectors unless noted).

A whole-vector 2-norm can hide a few wrong atoms (a row at a cell boundary,
a wrong periodic image), so every norm check in the parity tests has a
per-atom check beside it: the largest per-atom error, relative to the
largest per-atom value of the oracle vector (fields), or in Debye (dipoles).
"""
import numpy as np

DEBYE = 4.8032047


def rel(a, b):
    """2-norm of the difference over the 2-norm of b."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def max_atom_rel(a, b):
    """max_i |a_i - b_i| / max_i |b_i| (per-atom Euclidean norms)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b, axis=-1).max() / np.linalg.norm(b, axis=-1).max())


def rms_debye(a, b):
    """RMS over atoms of |a_i - b_i|, in Debye."""
    d = np.asarray(a) - np.asarray(b)
    return float(DEBYE * np.sqrt((d * d).sum() / d.shape[0]))


def max_atom_debye(a, b):
    """max_i |a_i - b_i| in Debye."""
    return float(DEBYE * np.linalg.norm(np.asarray(a) - np.asarray(b), axis=-1).max())


def assert_fields(a, b, tol, atom_factor=1.0):
    """2-norm relative error of a field below tol, per-atom below atom_factor * tol."""
    e, m = rel(a, b), max_atom_rel(a, b)
    assert e < tol and m < atom_factor * tol, f"2-norm {e:.3e}, per-atom {m:.3e} (tolerance {tol:g})"


def assert_dipoles(a, b, tol, atom_factor=1.0):
    """RMS dipole error below tol and the largest per-atom one below atom_factor * tol (Debye)."""
    e, m = rms_debye(a, b), max_atom_debye(a, b)
    assert e < tol and m < atom_factor * tol, f"RMS {e:.3e} D, per-atom {m:.3e} D (tolerance {tol:g})"

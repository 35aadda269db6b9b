"""The C-ABI library builds for sm_103a, loads, and exports every declared call.

These run without a GPU: they only load the shared library and look up
symbols; nothing computes.
"""
import ctypes
import os

import pytest

from paper_1906_01211_gb300 import build as build_mod


@pytest.fixture(scope="module")
def lib_path():
    return build_mod.build()


def test_library_exports_every_declared_function(lib_path):
    from paper_1906_01211_gb300 import amoebapol
    names = amoebapol.header_functions()
    assert {"amp_create", "amp_set_system", "amp_permanent_field", "amp_apply_T",
            "amp_solve_induced", "amp_polarization_energy", "amp_destroy"} <= set(names)
    lib = ctypes.CDLL(lib_path)
    for name in names:
        assert hasattr(lib, name), name


def test_create_rejects_bad_config(lib_path):
    from paper_1906_01211_gb300 import amoebapol as ap
    bad = [
        ap.Config(box=10.0, cutoff=7.0),                  # cutoff >= box/2
        ap.Config(box=30.0, pme_order=4),                 # order must be 5
        ap.Config(box=30.0, pme_grid=4),
        ap.Config(box=30.0, tol_debye=0.0),
    ]
    for cfg in bad:
        with pytest.raises(ap.AmpError) as e:
            ap.amp_create(cfg.to_c(), None)
        assert e.value.code == ap.AMP_ERR_ARG


def test_null_context_calls_fail_cleanly(lib_path):
    from paper_1906_01211_gb300 import amoebapol as ap
    assert ap._lib.amp_set_system(None, 3, None, None, None, None, None, None, None) == ap.AMP_ERR_ARG
    assert ap._lib.amp_multipole_energy(None, None, None, None, None, None) == ap.AMP_ERR_ARG
    assert ap.amp_last_error(None) == "null context"


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: loading the binding against a missing library raises."""
    import subprocess
    import sys
    code = ("import paper_1906_01211_gb300.amoebapol as ap, ctypes\n"
            "ap.LIB_PATH = %r\n"
            "try:\n    ap._load()\nexcept ImportError as e:\n    print('raised')\n") % str(tmp_path / "missing.so")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert "raised" in out.stdout, out.stderr


def test_predictor_coefficients(lib_path):
    """ASPC coefficients (Kolafa, J. Comput. Chem. 25, 335 (2004)): the values
    of orders 0..2 printed there, and for every order the two properties that
    make the predictor consistent: the coefficients sum to one and the
    predictor is exact on data linear in time (sum of -j B_j = 0)."""
    from fractions import Fraction as F
    from paper_1906_01211_gb300 import amoebapol as ap
    published = {0: [2, -1], 1: [F(5, 2), -2, F(1, 2)], 2: [F(14, 5), F(-14, 5), F(6, 5), F(-1, 5)]}
    for k, want in published.items():
        got = ap.amp_predictor_coefficients(k)
        assert len(got) == k + 2
        assert all(abs(g - float(w)) < 1e-14 for g, w in zip(got, want))
    for k in range(7):
        b = ap.amp_predictor_coefficients(k)
        assert abs(sum(b) - 1.0) < 1e-13
        assert abs(sum(-(j + 1) * bj for j, bj in enumerate(b))) < 1e-12
    with pytest.raises(ap.AmpError):
        ap.amp_predictor_coefficients(7)

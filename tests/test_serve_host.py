"""Serving layer on the host, without a GPU: the binding's structures against
the header, the server's argument checks (which run before any CUDA call),
and the seeded request stream. The server itself runs on the GPU
(tests/test_gpu_serving.py); failures there are made on the host (invalid
requests, a request larger than the budget), never on a GPU."""
import ctypes
import re

import numpy as np
import pytest

from paper_1906_01211_gb300.serve import percentile, request_stream


def header_struct_fields(name):
    from paper_1906_01211_gb300.amoebapol import HEADER_PATH
    text = open(HEADER_PATH).read()
    structs = {nm: body for body, nm in re.findall(r"typedef struct \{([^}]*)\}\s*(\w+);", text)}
    assert name in structs, name
    body = re.sub(r"/\*.*?\*/", "", structs[name], flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = re.match(r"((?:const\s+)?(?:long long|unsigned|int|double|char))\s+(.*)", decl).groups()
        for nm in names.split(","):
            nm = nm.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", nm)
            fields.append((arr.group(1), ctype, int(arr.group(2))) if arr else (nm, ctype, 1))
    return fields


CTYPES = {"int": ctypes.c_int, "long long": ctypes.c_longlong, "double": ctypes.c_double, "char": ctypes.c_char}


@pytest.mark.parametrize("name", ["amp_server_config", "amp_server_result", "amp_server_counters"])
def test_binding_structs_match_header(name):
    from paper_1906_01211_gb300 import amoebapol as ap
    cls = getattr(ap, name)
    want = header_struct_fields(name)
    got = cls._fields_
    assert [f[0] for f in got] == [w[0] for w in want]
    for (fname, ftype), (_, ctype, count) in zip(got, want):
        base = CTYPES[ctype]
        assert ftype == (base * count if count > 1 else base), fname


def test_server_rejects_bad_configuration_before_touching_the_device():
    from paper_1906_01211_gb300 import amoebapol as ap
    bad = [dict(n_workers=0), dict(mem_budget_bytes=0), dict(tol_debye=0.0), dict(max_iter=0), dict(precision=7),
           dict(batch_max_atoms=100, batch_arena_atoms=50), dict(batch_max_atoms=100, batch_max_requests=0),
           dict(resident_bytes=-1)]
    base = dict(n_workers=2, mem_budget_bytes=1 << 30, precision=ap.AMP_MIXED, tol_debye=1e-5, max_iter=100,
                batch_max_atoms=0, batch_arena_atoms=0, batch_max_requests=0, resident_bytes=0)
    for b in bad:
        cfg = ap.amp_server_config(**{**base, **b})
        h = ctypes.c_void_p()
        assert ap._lib.amp_server_create(ctypes.byref(h), ctypes.byref(cfg), 0) == ap.AMP_ERR_ARG
        assert not h.value
    assert ap._lib.amp_server_create(None, None, 0) == ap.AMP_ERR_ARG


def test_server_calls_reject_null_arguments():
    from paper_1906_01211_gb300 import amoebapol as ap
    t = ctypes.c_longlong(0)
    z = np.zeros(6)
    m = np.zeros(2, dtype=np.int32)
    args = [z.ctypes.data] * 6 + [m.ctypes.data]
    assert ap._lib.amp_server_submit(None, 2, 0.0, 0.0, 0.0, 0, *args, None, ctypes.byref(t)) == ap.AMP_ERR_ARG
    assert ap._lib.amp_server_poll(None, 0, None, None) == ap.AMP_ERR_ARG
    assert ap._lib.amp_server_wait(None, 0, 0.0, None, None) == ap.AMP_ERR_ARG
    assert ap._lib.amp_server_stats(None, None) == ap.AMP_ERR_ARG
    ap._lib.amp_server_destroy(None)  # ignored


def test_request_stream_is_seeded_and_mixed():
    a = request_stream(40, seed=4)
    b = request_stream(40, seed=4)
    assert [s.n for s in a] == [s.n for s in b]
    assert np.array_equal(a[5].xyz, b[5].xyz)
    sizes = np.array([s.n // 3 for s in a])
    assert sizes.min() >= 64 and sizes.max() <= 4096
    kinds = [s.box is None for s in a]
    assert 0 < sum(kinds) < len(kinds)


def test_percentile():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    with pytest.raises(TypeError):
        percentile(None, 50)

"""The package's DC-JI block partition (host logic, no GPU) against the
oracle's reading: whole molecules, each to the cell of its first site, empty
cells dropped, blocks in cell order (oracle/dcji.py)."""
import importlib.util
import os

import numpy as np
import pytest

from oracle.dcji import cell_blocks as oracle_blocks
from paper_1906_01211_gb300.synth import density_box_edge, make_waters


def _package_cell_blocks():
    # the helper is plain numpy; load it without the CUDA library
    path = os.path.join(os.path.dirname(__file__), "..", "paper_1906_01211_gb300", "amoebapol.py")
    src = open(path).read()
    ns = {}
    exec(src[src.index("def cell_blocks"):src.index("def amp_multipole_energy")], ns)
    return ns["cell_blocks"]


@pytest.mark.parametrize("nw,periodic,cells", [(64, True, 1), (64, True, 2), (64, True, 4), (60, False, 3)])
def test_partition_matches_the_oracle(nw, periodic, cells):
    s = make_waters(nw, density_box_edge(nw), 5, periodic=periodic)
    block_of, nb = _package_cell_blocks()(s.xyz, s.mol, s.box if s.box is not None else 0.0, cells)
    ref = oracle_blocks(s, cells)
    assert nb == len(ref)
    for b, r in enumerate(ref):
        assert np.array_equal(np.flatnonzero(block_of == b), r)

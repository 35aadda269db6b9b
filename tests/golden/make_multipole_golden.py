"""Writes multipole_water23556.json: the oracle's permanent-multipole energy of
the 23,556-atom water box and its gradients at eight sampled atoms.

Run from the repository root: python tests/golden/make_multipole_golden.py
Only the oracle computes the values; the inputs come from the seeded generator.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import Setup  # noqa: E402
from oracle.multipole import multipole_energy, multipole_rows  # noqa: E402
from paper_1906_01211_gb300.synth import WATER_23556  # noqa: E402


def main():
    w = WATER_23556
    s = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    rows = np.random.Generator(np.random.PCG64(11)).choice(s.n, 8, replace=False)
    U = multipole_energy(s, st, with_gradients=False)
    F, gq, gd, gt = multipole_rows(s, st, rows)
    out = {"workload": w.name, "U_kcal_mol": U, "rows": [int(r) for r in rows],
           "F": F.tolist(), "gq": gq.tolist(), "gd": gd.tolist(), "gquad": gt.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "multipole_water23556.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()

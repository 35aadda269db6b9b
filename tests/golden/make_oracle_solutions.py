"""Writes water23556_oracle.npz and water96000_oracle.npz: the oracle's
solutions of the 23,556-atom (DHFR-sized) and 96,000-atom (Puddle-sized)
water boxes, the two large workloads of the paper's Section "Execution
setup".

Stored per box: the oracle's permanent field E0 (float64, [N][3]); the
induced dipoles mu, energy U and iteration count of the oracle's PCG run to
1e-8 D RMS preconditioned residual (mu, U, iters); the same for the run to
the box's own tolerance, 1e-5 D (mu_tol, U_tol, iters_tol); the unique pair
count. The GPU tests hold the 96,000-atom float64 solve (run to 1e-8 D) to
the first and the mixed solve (run to 1e-5 D) to the second; the benchmark
reports both precisions' errors against them.

Run from the repository root: python tests/golden/make_oracle_solutions.py
Only the oracle computes the values; the inputs come from the seeded
generator. Takes about two minutes on one core.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import Setup  # noqa: E402
from oracle.energy import polarization_energy  # noqa: E402
from oracle.solver import Operator, solve  # noqa: E402
from paper_1906_01211_gb300.synth import WATER_23556, WATER_96000  # noqa: E402

TOL_DEBYE = 1e-8
HERE = os.path.dirname(os.path.abspath(__file__))


def path_for(name: str) -> str:
    return os.path.join(HERE, name.replace("-", "") + "_oracle.npz")


def write(w):
    s = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    t0 = time.time()
    op = Operator(s, st)
    E0 = op.permanent_field()
    mu, iters, rms = solve(op, E0, TOL_DEBYE)
    U = polarization_energy(mu, E0)
    mu_t, iters_t, rms_t = solve(op, E0, w.tol_debye)
    U_t = polarization_energy(mu_t, E0)
    np.savez_compressed(path_for(w.name), workload=w.name, tol_debye=TOL_DEBYE, mu=mu, E0=E0, U=U, iters=iters,
                        rms=rms, tol_box=w.tol_debye, mu_tol=mu_t, U_tol=U_t, iters_tol=iters_t,
                        n_pairs=op.n_pairs)
    print(f"{w.name}: {op.n_pairs} pairs; {iters} iterations to {TOL_DEBYE:g} D (rms {rms:.3e}), U = {U!r}; "
          f"{iters_t} iterations to {w.tol_debye:g} D, U = {U_t!r} ({time.time() - t0:.0f} s)")


def main():
    for w in (WATER_23556, WATER_96000):
        write(w)


if __name__ == "__main__":
    main()

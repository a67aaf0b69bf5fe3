"""Writes oracle-only reference values used by the parity tests and by the
CPU baseline: the converged free energy of the 64-H r_s=2 theta=1 cell on
128^3 (and of the fcc cell on 32^3), computed by oracle/ alone.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.functional import Functional  # noqa: E402
from oracle.minimize import lbfgs  # noqa: E402
from workloads import config_cell  # noqa: E402


def main():
    out = {}
    for idx, tolF, tolR in ((1, 1e-11, 1e-8), (2, 1e-9, 1e-6)):
        cell = config_cell(idx)
        t0 = time.time()
        F = Functional(cell)
        t_setup = time.time() - t0
        r = lbfgs(F, tol_F=tolF, tol_R=tolR, max_iter=2000)
        out[cell.label] = dict(energies=r.energies, iterations=r.iterations, evaluations=r.evaluations,
                               converged=r.converged, tol_F_per_ion=tolF, tol_residual=tolR,
                               setup_seconds=t_setup, minimise_seconds=time.time() - t0 - t_setup,
                               n=cell.n, n_ion=cell.n_ion)
        print(cell.label, out[cell.label], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_minima.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()

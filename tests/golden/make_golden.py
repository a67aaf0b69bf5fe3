"""Writes oracle-only reference values used by the parity tests and by the
CPU baseline, computed by oracle/ alone:

* fcc4_Z3_n32: the converged minimum of the fcc cell on 32^3 (plain L-BFGS);
* rand64_H_rs2_n128: the converged minimum of the 64-H r_s=2 theta=1 cell on
  128^3 (plain L-BFGS: energies and evaluation count), and the same minimum
  reached with the oracle's preconditioner, whose density is stored as
  float32 in oracle_density_rand64_H_rs2_n128.npy;
* rand1024_Z3_rs2.5_n256: the converged minimum of the 1024-ion cell on 256^3
  (preconditioned L-BFGS; a plain run would take hours on a CPU).

Entries are merged into oracle_minima.json; name the ones to (re)compute,
e.g.  python tests/golden/make_golden.py rand1024_Z3_rs2.5_n256
(no argument: all of them).  Run from the repository root.
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from oracle.functional import Functional  # noqa: E402
from oracle.minimize import lbfgs  # noqa: E402
from workloads import config_cell  # noqa: E402

JSON = os.path.join(HERE, "oracle_minima.json")


def precond_args(cell):
    """The oracle's preconditioner: c = 4 (E_F + T) at the mean density, with
    the kernel's curvature and 1.5 times the Hartree term."""
    kF = (3 * math.pi ** 2 * cell.n_electrons / cell.volume) ** (1 / 3)
    return dict(precond_c=4 * (0.5 * kF ** 2 + cell.T), precond_k=1.0, precond_h=1.5)


def run(idx, tolF, tolR, precond):
    cell = config_cell(idx)
    t0 = time.time()
    F = Functional(cell)
    t_setup = time.time() - t0
    kw = precond_args(cell) if precond else {}
    r = lbfgs(F, tol_F=tolF, tol_R=tolR, max_iter=4000, **kw)
    entry = dict(energies=r.energies, iterations=r.iterations, evaluations=r.evaluations,
                 converged=r.converged, tol_F_per_ion=tolF, tol_residual=tolR,
                 setup_seconds=t_setup, minimise_seconds=time.time() - t0 - t_setup,
                 n=cell.n, n_ion=cell.n_ion, preconditioned=bool(precond))
    return cell, r, entry


def main(which):
    out = {}
    if os.path.exists(JSON):
        with open(JSON) as f:
            out = json.load(f)

    def want(label):
        return not which or label in which

    if want("fcc4_Z3_n32"):
        cell, _, e = run(1, 1e-11, 1e-8, False)
        out[cell.label] = e
    if want("rand64_H_rs2_n128"):
        cell, _, e = run(2, 1e-9, 1e-6, False)
        out[cell.label] = e
    if want("rand64_H_rs2_n128_precond"):
        cell, r, e = run(2, 1e-9, 1e-6, True)
        out[cell.label + "_precond"] = e
        np.save(os.path.join(HERE, f"oracle_density_{cell.label}.npy"), r.rho.astype(np.float32))
    if want("rand1024_Z3_rs2.5_n256"):
        cell, _, e = run(4, 1e-8, 1e-5, True)
        out[cell.label] = e
    for k, v in out.items():
        print(k, {kk: vv for kk, vv in v.items() if kk != "energies"}, flush=True)
    with open(JSON, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(set(sys.argv[1:]))

"""Pressure P = -dF/dOmega (Results: Table 1, Fig. 3) from the CUDA path,
through the C-ABI, against the FP64 oracle (oracle/pressure.py, pinned per term
to energy differences on dilated cells).

Tolerances, per term, relative to the largest term: FP64 plans 1e-9 (the
kernel-derivative table is a difference quotient of two independently
integrated Lindhard kernels, which amplifies their ~1e-13 quadrature
differences by ~1e3); FP32 plans 2e-5 (single-precision pointwise TF/xc and
transforms, compensated sums)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.pressure import pressure as oracle_pressure
from workloads import random_cell, config_cell, SEED_BASE
from workloads.cells import Cell
import paper_2601_23002_gb300 as og

from test_gpu_parity import rand_density

CELLS = [("h24", lambda: random_cell(SEED_BASE + 11, 9, 1.0, 1.8, 0.9, 24)),
         ("z4_40", lambda: random_cell(SEED_BASE + 12, 5, 4.0, 1.6, 0.4, 40)),
         ("z3_50", lambda: random_cell(SEED_BASE + 13, 7, 3.0, 2.1, 1.3, 50))]
TOL = {"fp64": 1e-9, "fp32": 2e-5}
KEYS = ("tf", "vw", "nl", "hartree", "loc", "xc", "ion", "total")


def _compare(got, ref, tol, label):
    scale = max(abs(ref[k]) for k in KEYS)
    for k in KEYS:
        print(f"{label} {k}: gpu {got[k]:.12e} oracle {ref[k]:.12e}")
        assert abs(got[k] - ref[k]) < tol * scale, (label, k, got[k], ref[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", CELLS)
def test_pressure_matches_oracle(name, mk, precision):
    cell = mk()
    rho = rand_density(cell, 31)
    ref = oracle_pressure(cell, rho)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    got = plan.pressure(torch.tensor(rho, dtype=dt, device="cuda").reshape(-1))
    plan.close()
    _compare(got, ref, TOL[precision], f"{name} {precision}")


def test_pressure_wang_teter_exponent():
    # a = 5/6: the (3 - 6a) K part of the NL term no longer vanishes
    cell = CELLS[0][1]()
    rho = rand_density(cell, 32)
    ref = oracle_pressure(cell, rho, alpha=5.0 / 6.0)
    plan = og.plan_for_cell(cell, alpha=5.0 / 6.0)
    got = plan.pressure(torch.tensor(rho, device="cuda").reshape(-1))
    plan.close()
    _compare(got, ref, TOL["fp64"], "h24 a=5/6")


def test_pressure_with_terms_off():
    cell = CELLS[1][1]()
    rho = rand_density(cell, 33)
    terms = og.TERM_TF | og.TERM_VW | og.TERM_HARTREE
    ref = oracle_pressure(cell, rho, terms=("tf", "vw", "hartree"))
    plan = og.plan_for_cell(cell, terms=terms)
    got = plan.pressure(torch.tensor(rho, device="cuda").reshape(-1))
    plan.close()
    assert got["nl"] == 0.0 and got["loc"] == 0.0 and got["xc"] == 0.0
    _compare(got, ref, TOL["fp64"], "z4_40 tf+vw+H")


def _dilated(cell, lam):
    return Cell(L=cell.L * lam, n=cell.n, Z=cell.Z, pos=np.asarray(cell.pos) * lam,
                theta=cell.theta * lam * lam, rc=cell.rc, label=cell.label)


def test_full_size_128_pressure_at_the_minimum():
    # 64 H at r_s = 2 on 128^3, the launch the benchmark times: the GPU
    # pressure at the GPU minimum against the oracle at that density, and
    # against -dF_min/dOmega from minima of the dilated cells (at the minimum
    # the path of n does not matter: the virial pressure is the derivative of
    # the minimised free energy)
    cell = config_cell(2)
    fmin = {}
    for lam in (1.0, 1.001, 0.999):
        c = _dilated(cell, lam)
        plan = og.plan_for_cell(c)
        rho = torch.empty(c.n ** 3, dtype=torch.float64, device="cuda")
        out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=1e-11, tol_residual=1e-7)
        assert out["converged"], out
        fmin[lam] = out["F_total"]
        if lam == 1.0:
            got = plan.pressure(rho)
            n_np = rho.cpu().numpy().reshape((c.n,) * 3)
        plan.close()
    ref = oracle_pressure(cell, n_np)
    _compare(got, ref, TOL["fp64"], "rand64H 128")
    dF = (fmin[1.001] - fmin[0.999]) / (2 * 1e-3)
    p_fd = -dF / (3 * cell.volume)
    print(f"virial {got['total']:.10e}  -dFmin/dOmega {p_fd:.10e}")
    # central-difference error O(1e-6) relative plus the minima's convergence
    assert abs(got["total"] - p_fd) < 1e-5 * abs(got["total"]) + 64 * 1e-11 / (2e-3 * 3 * cell.volume)

"""Hellmann-Feynman forces on the ions (Methods: the forces of the molecular
dynamics that produces the structure factors) from the CUDA path, through the
C-ABI, against the FP64 oracle (oracle/forces.py, itself pinned to finite
differences of the oracle energy).

The GPU sums the local and reciprocal Ewald terms over the half spectrum with
|G|^2 <= 156/rc^2 (form factors below exp(-39) beyond), the oracle over the
whole grid; the cells here keep that sphere inside the grid, so both sums
agree to rounding.  Tolerances: FP64 plans 1e-9 of max|F| (rounding only);
FP32 plans 2e-5 of max|F| (single-precision transform of n and phases, each
term rounded at ~1e-7 of its size, compensated sums over ~1e4 terms)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.forces import forces as oracle_forces, local_forces, ewald_forces
from workloads import random_cell, config_cell, SEED_BASE
import paper_2601_23002_gb300 as og

from test_gpu_parity import rand_density

CELLS = [("h24", lambda: random_cell(SEED_BASE + 11, 9, 1.0, 1.8, 0.9, 24)),
         ("z4_40", lambda: random_cell(SEED_BASE + 12, 5, 4.0, 1.6, 0.4, 40)),
         ("z3_50", lambda: random_cell(SEED_BASE + 13, 7, 3.0, 2.1, 1.3, 50))]
TOL = {"fp64": 1e-9, "fp32": 2e-5}


def gpu_forces(cell, rho, precision):
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    f = plan.forces(torch.tensor(rho, dtype=dt, device="cuda").reshape(-1))
    plan.close()
    return f


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", CELLS)
def test_forces_match_oracle(name, mk, precision):
    cell = mk()
    rho = rand_density(cell, 21)
    ref = oracle_forces(cell, rho)
    got = gpu_forces(cell, rho, precision)
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print(f"{name} {precision}: max|F| {scale:.3e} max err {err:.3e}")
    assert err < TOL[precision] * scale


def test_forces_without_local_term_are_ewald_only():
    cell = CELLS[0][1]()
    rho = rand_density(cell, 22)
    terms = og.TERMS_ALL & ~og.TERM_LOC
    plan = og.plan_for_cell(cell, terms=terms)
    f = plan.forces(torch.tensor(rho, device="cuda").reshape(-1))
    plan.close()
    ref = ewald_forces(np.asarray(cell.Z, float), cell.pos, cell.L)
    assert np.abs(f - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(ref).max()


def test_forces_are_the_derivative_of_the_gpu_energy():
    # central differences of the plan's own energy at fixed rho, ions moved
    cell = CELLS[2][1]()
    rho = torch.tensor(rand_density(cell, 23), device="cuda").reshape(-1)
    plan = og.plan_for_cell(cell)
    f = plan.forces(rho)
    h = 1e-4
    for I, d in ((0, 0), (3, 1), (6, 2)):
        e = []
        for s in (+1, -1):
            pos = np.array(cell.pos, float).copy()
            pos[I, d] += s * h
            plan.structure_factor(pos)
            e.append(plan.energy_potential(rho)["F_total"])
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - f[I, d]) < 1e-6 * max(1.0, abs(f[I, d])), (I, d, fd, f[I, d])
    plan.close()


def test_forces_before_structure_factor_is_an_error():
    cell = CELLS[0][1]()
    plan = og.Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc)
    with pytest.raises(og.OfdftError):
        plan.forces(torch.ones(cell.n ** 3, dtype=torch.float64, device="cuda"))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_128_forces_at_the_minimum(precision):
    # 64 H at r_s = 2 on 128^3, the launch the benchmark times: forces at the
    # GPU minimum against the oracle for sampled ions (the oracle's local
    # force of one ion needs only that ion), and the net force.  Translating
    # every ion by delta is translating n by -delta, under which all terms but
    # E_loc are invariant, so sum_I F_I = -int (v - mu) grad n; Cauchy-Schwarz
    # with R^2 = int n (v - mu)^2 / N_e and E_vW = (1/8) int |grad n|^2 / n
    # bounds it by R sqrt(8 N_e E_vW) per component.
    cell = config_cell(2)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
    if precision == "fp64":
        out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=1e-9, tol_residual=1e-6)
    else:
        out = plan.minimize(rho, start_uniform=True)
    assert out["converged"], out
    f = plan.forces(rho)
    plan.close()
    n_np = rho.double().cpu().numpy().reshape((cell.n,) * 3)
    Z = np.asarray(cell.Z, float)
    pos = np.asarray(cell.pos, float)
    sel = np.array([0, 17, 40, 63])
    ref = local_forces(Z[sel], pos[sel], n_np, cell.L, cell.rc) + ewald_forces(Z, pos, cell.L)[sel]
    scale = np.abs(ref).max()
    err = np.abs(f[sel] - ref).max()
    net = np.abs(f.sum(axis=0)).max()
    bound = out["residual"] * np.sqrt(8.0 * cell.n_electrons * out["E_vW"])
    print(f"{precision}: max|F| {scale:.3e} max err {err:.3e} |sum F| {net:.3e} bound {bound:.3e}")
    assert err < TOL[precision] * scale
    assert net < 1.5 * bound + TOL[precision] * scale

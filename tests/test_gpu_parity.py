"""CUDA path (through the C-ABI) against the FP64 CPU oracle, element by
element on seeded inputs.  Tolerances: FP64 plans to 1e-9 Ha/ion in energy
and 1e-8 Ha in the potential (rounding only); FP32-bulk plans to 1e-5 Ha/ion
and 1e-4 relative in the potential (single-precision FFTs and pointwise
terms, FP64 sums).  Minimisation parity: 1e-6 Ha/ion in F and 1e-5 relative
L2 in n (both sides converged to tight tolerances)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.functional import Functional
from oracle.minimize import lbfgs
from oracle.sei import sei_shells as oracle_sei
from oracle.cell import structure_factor as oracle_sf
from workloads import fcc_cell, random_cell, config_cell, SEED_BASE
import paper_2601_23002_gb300 as og

TERMS = {"tf": og.TERM_TF, "vw": og.TERM_VW, "nl": og.TERM_NL, "xc": og.TERM_XC,
         "hartree": og.TERM_HARTREE, "loc": og.TERM_LOC}


def rand_density(cell, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    n = cell.n
    nbar = cell.n_electrons / cell.volume
    x = np.arange(n) / n
    smooth = sum(rng.uniform(0.2, 1.0) * np.cos(2 * math.pi * (k[0] * x[:, None, None] + k[1] * x[None, :, None]
                                                                + k[2] * x[None, None, :]) + rng.uniform(0, 6.28))
                 for k in rng.integers(-3, 4, size=(6, 3)))
    rho = nbar * np.exp(amp * smooth / 3.0)
    return rho * cell.n_electrons / (rho.sum() * cell.volume / rho.size)


def gpu_eval(cell, rho, precision="fp64", terms=og.TERMS_ALL, alpha=0.5):
    plan = og.plan_for_cell(cell, precision=precision, terms=terms, alpha=alpha)
    dt = torch.float32 if precision == "fp32" else torch.float64
    r = torch.tensor(rho, dtype=dt, device="cuda")
    v = torch.empty_like(r)
    e = plan.energy_potential(r, v)
    out = v.double().cpu().numpy()
    plan.close()
    return e, out


CASES = [("fcc16", lambda: fcc_cell(n=16)),
         ("fcc32", lambda: fcc_cell(n=32)),
         ("h24", lambda: random_cell(SEED_BASE + 11, 9, 1.0, 1.8, 0.9, 24)),
         ("z4_40", lambda: random_cell(SEED_BASE + 12, 5, 4.0, 1.6, 0.4, 40)),
         ("z3_50", lambda: random_cell(SEED_BASE + 13, 7, 3.0, 2.1, 1.3, 50)),
         ("h54", lambda: random_cell(SEED_BASE + 14, 12, 1.0, 2.0, 1.0, 54))]


@pytest.mark.parametrize("name,mk", CASES)
def test_energy_potential_fp64(name, mk):
    cell = mk()
    rho = rand_density(cell, 1)
    e, v = gpu_eval(cell, rho)
    ref_e, ref_v = Functional(cell).evaluate(rho)
    ni = cell.n_ion
    assert abs(e["F_total"] - ref_e["total"]) / ni < 1e-9
    for k_gpu, k_ref in (("F_TF", "tf"), ("E_vW", "vw"), ("E_NL", "nl"), ("E_H", "hartree"),
                         ("E_loc", "loc"), ("E_xc", "xc"), ("E_ion", "ion")):
        assert abs(e[k_gpu] - ref_e[k_ref]) < 1e-9 * max(1.0, abs(ref_e[k_ref])), (k_gpu, e[k_gpu], ref_e[k_ref])
    assert abs(e["N_e"] - cell.n_electrons) < 1e-10 * cell.n_electrons
    assert abs(e["mu"] - ref_e["mu"]) < 1e-9
    assert np.max(np.abs(v - ref_v)) < 1e-8 * max(1.0, np.max(np.abs(ref_v)))


@pytest.mark.parametrize("term", list(TERMS))
def test_each_term_alone_fp64(term):
    cell = random_cell(SEED_BASE + 21, 6, 3.0, 1.7, 0.6, 24)
    rho = rand_density(cell, 2)
    e, v = gpu_eval(cell, rho, terms=TERMS[term])
    ref_e, ref_v = Functional(cell, terms=(term,)).evaluate(rho)
    assert abs(e["F_total"] - ref_e["total"]) < 1e-9 * max(1.0, abs(ref_e["total"]))
    assert np.max(np.abs(v - ref_v)) < 1e-8 * max(1.0, np.max(np.abs(ref_v)))


def test_wang_teter_exponent_option():
    cell = random_cell(SEED_BASE + 22, 8, 1.0, 2.0, 1.0, 32)
    rho = rand_density(cell, 3)
    e, v = gpu_eval(cell, rho, alpha=5 / 6)
    ref_e, ref_v = Functional(cell, alpha=5 / 6).evaluate(rho)
    assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < 1e-9
    assert np.max(np.abs(v - ref_v)) < 1e-8 * max(1.0, np.max(np.abs(ref_v)))


@pytest.mark.parametrize("name,mk", CASES)
def test_energy_potential_fp32(name, mk):
    cell = mk()
    rho = rand_density(cell, 4)
    e, v = gpu_eval(cell, rho, precision="fp32")
    rho32 = rho.astype(np.float32).astype(np.float64)
    ref_e, ref_v = Functional(cell).evaluate(rho32)
    assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < 1e-5
    assert np.max(np.abs(v - ref_v)) < 1e-4 * max(1.0, np.max(np.abs(ref_v)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,mk", [CASES[2], CASES[4]])
def test_plane_and_tiled_paths_match_oracle(precision, name, mk, monkeypatch):
    """Grids whose kz planes fit in shared memory take the fused plane pass;
    OFDFT_PLANE=0 forces the tiled y / x-G-space / y chain.  Both against the
    oracle, and against each other (same arithmetic, other FFT factorisation
    and summation order)."""
    cell = mk()
    rho = rand_density(cell, 5)
    if precision == "fp32":
        rho = rho.astype(np.float32).astype(np.float64)
    ref_e, ref_v = Functional(cell).evaluate(rho)
    e1, v1 = gpu_eval(cell, rho, precision=precision)
    monkeypatch.setenv("OFDFT_PLANE", "0")
    e2, v2 = gpu_eval(cell, rho, precision=precision)
    tol_e, tol_v = (1e-9, 1e-8) if precision == "fp64" else (1e-5, 1e-4)
    vmax = max(1.0, np.max(np.abs(ref_v)))
    for e, v in ((e1, v1), (e2, v2)):
        assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < tol_e
        assert np.max(np.abs(v - ref_v)) < tol_v * vmax
    assert abs(e1["F_total"] - e2["F_total"]) / cell.n_ion < tol_e
    assert np.max(np.abs(v1 - v2)) < tol_v * vmax


def test_structure_factor_matches_oracle():
    cell = random_cell(SEED_BASE + 31, 17, 1.0, 1.9, 1.0, 24)
    plan = og.Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc)
    S = torch.empty((24, 24, 13), dtype=torch.complex128, device="cuda")
    plan.structure_factor(cell.pos, S_out=S)
    ref = oracle_sf(cell.pos, 24, cell.L)[:, :, :13]
    assert np.max(np.abs(S.cpu().numpy() - ref)) < 1e-11
    plan.close()


def test_sei_shells_match_oracle():
    cell = random_cell(SEED_BASE + 32, 10, 1.0, 2.0, 1.0, 32)
    rho = rand_density(cell, 5)
    plan = og.plan_for_cell(cell)
    q, s = plan.sei_shells(torch.tensor(rho, device="cuda"), 60)
    qr, sr = oracle_sei(rho, cell.pos, cell.L, cell.n_electrons, 60)
    assert np.allclose(q, qr, rtol=1e-14)
    assert np.max(np.abs(s - sr)) < 1e-10
    plan.close()


def test_errors_are_reported_not_faulted():
    cell = fcc_cell(n=16)
    plan = og.Plan(cell.L, cell.n, cell.Z, cell.T)
    r = torch.ones(16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(og.OfdftError):
        plan.energy_potential(r)            # no structure factor yet
    with pytest.raises(ValueError):
        plan.energy_potential(torch.ones(10, dtype=torch.float64, device="cuda"))
    plan.close()


# ------------------------------------------------------------------ minimiser
@pytest.fixture(scope="module")
def fcc_oracle_min():
    cell = config_cell(1)
    F = Functional(cell)
    r = lbfgs(F, tol_F=1e-11, tol_R=1e-8, max_iter=800)
    assert r.converged
    return cell, r


def test_minimize_fp64_matches_oracle(fcc_oracle_min):
    cell, ref = fcc_oracle_min
    plan = og.plan_for_cell(cell, precision="fp64")
    rho = torch.empty(cell.n ** 3, dtype=torch.float64, device="cuda")
    out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=1e-11, tol_residual=1e-8, max_iter=800)
    assert out["converged"], out
    n_gpu = rho.cpu().numpy().reshape((cell.n,) * 3)
    assert abs(out["F_total"] - ref.energies["total"]) / cell.n_ion < 1e-6
    assert np.linalg.norm(n_gpu - ref.rho) / np.linalg.norm(ref.rho) < 1e-5
    assert abs(n_gpu.sum() * cell.volume / n_gpu.size - cell.n_electrons) < 1e-10 * cell.n_electrons
    # deterministic
    rho2 = torch.empty_like(rho)
    out2 = plan.minimize(rho2, start_uniform=True, tol_F_per_ion=1e-11, tol_residual=1e-8, max_iter=800)
    assert torch.equal(rho, rho2) and out2["F_total"] == out["F_total"]
    plan.close()


def test_minimize_fp32_error_against_fp64_oracle(fcc_oracle_min):
    cell, ref = fcc_oracle_min
    plan = og.plan_for_cell(cell, precision="fp32")
    rho = torch.empty(cell.n ** 3, dtype=torch.float32, device="cuda")
    out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=1e-7, tol_residual=1e-5, max_iter=800)
    n_gpu = rho.double().cpu().numpy().reshape((cell.n,) * 3)
    dF = abs(out["F_total"] - ref.energies["total"]) / cell.n_ion
    dn = np.linalg.norm(n_gpu - ref.rho) / np.linalg.norm(ref.rho)
    print(f"fp32 vs fp64 oracle: |dF|/ion = {dF:.2e}, rel L2 density = {dn:.2e}")
    assert dF < 1e-6
    assert dn < 1e-4
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_128_minimum_is_oracle_stationary(precision):
    # 64 H at r_s = 2 on 128^3: the GPU minimum, re-evaluated by the oracle at
    # the same density, has the same free energy and a small Euler-Lagrange
    # residual (a property of the minimum that holds at any size)
    cell = config_cell(2)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
    out = plan.minimize(rho, start_uniform=True)
    assert out["converged"], out
    n_gpu = rho.double().cpu().numpy().reshape((cell.n,) * 3)
    F = Functional(cell)
    psi = np.sqrt(n_gpu)
    e, g, _ = F.evaluate_psi(psi)
    tol = 1e-6 if precision == "fp64" else 1e-5
    assert abs(e["total"] - out["F_total"]) / cell.n_ion < tol
    assert e["residual"] < 3e-4
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_128_matches_converged_oracle(precision):
    # the oracle's own converged minimum of the 64-H 128^3 cell (written by
    # tests/golden/make_golden.py from oracle/ alone) against the GPU minimum
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_minima.json")) as f:
        ref = json.load(f)["rand64_H_rs2_n128"]
    cell = config_cell(2)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
    out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=1e-9, tol_residual=1e-6 if precision == "fp64" else 2e-5)
    plan.close()
    dF = abs(out["F_total"] - ref["energies"]["total"]) / cell.n_ion
    print(f"{precision}: |F_gpu - F_oracle|/ion = {dF:.2e}")
    assert dF < 1e-6


def test_full_size_256_1024_ions_terms_and_sei():
    # 1024 Z=3 ions at r_s = 2.5, theta = 0.3 on 256^3, FP32 bulk (the largest
    # single-cell workload): the GPU minimum converges with N_e exact; at that
    # density the terms the oracle can form at this size (pointwise TF and XC,
    # Hartree and vW by one transform each, Ewald) agree to 1e-5 Ha/ion, and
    # S_ei on the first 200 shells agrees with the oracle's direct sum.
    from oracle import fermi_dirac as fd, xc as oxc
    from oracle.cell import ewald_energy, g2_grid
    from oracle.functional import fft3, N_MIN
    from oracle.sei import sei_shells_direct
    cell = config_cell(4)
    plan = og.plan_for_cell(cell, precision="fp32")
    rho = torch.empty(cell.n ** 3, dtype=torch.float32, device="cuda")
    out = plan.minimize(rho, start_uniform=True)
    assert out["converged"], out
    assert abs(out["N_e"] - cell.n_electrons) < 1e-4 * cell.n_electrons
    q, s = plan.sei_shells(rho, 200)
    plan.close()
    n_np = rho.double().cpu().numpy().reshape((cell.n,) * 3)
    del rho
    Om, N, T = cell.volume, cell.n ** 3, cell.T
    dV = Om / N
    nf = np.maximum(n_np, N_MIN)
    f, _, _ = fd.tf_free_energy_density(nf, T)
    exc, _ = oxc.lda_xc(nf)
    nt = fft3(n_np)
    G2 = g2_grid(cell.n, cell.L)
    with np.errstate(divide="ignore", invalid="ignore"):
        coul = np.where(G2 > 0, 4 * math.pi / np.where(G2 > 0, G2, 1.0), 0.0)
    ref = {"F_TF": dV * float(np.sum(f)), "E_xc": dV * float(np.sum(n_np * exc)),
           "E_H": 0.5 * Om * float(np.sum(coul * np.abs(nt) ** 2)),
           "E_vW": 0.5 * Om * float(np.sum(G2 * np.abs(fft3(np.sqrt(n_np))) ** 2)),
           "E_ion": ewald_energy(np.asarray(cell.Z, float), cell.pos, cell.L)}
    del nt, G2, coul
    for k, v in ref.items():
        print(f"{k}: gpu {out[k]:.8f} oracle {v:.8f}")
        assert abs(out[k] - v) / cell.n_ion < 1e-5, k
    qr, sr = sei_shells_direct(n_np, cell.pos, cell.L, cell.n_electrons, 200)
    assert np.allclose(q, qr, rtol=1e-12)
    print("S_ei max |diff|", np.abs(s - sr).max(), "max |S|", np.abs(sr).max())
    assert np.abs(s - sr).max() < 1e-4 * max(1.0, np.abs(sr).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_async_energies_equal_the_synchronous_ones(precision):
    # ofdft_energy_potential_async forms the energies on the device; queued
    # back to back on one stream they match the synchronous call's
    cell = CASES[2][1]()
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rhos = [torch.tensor(rand_density(cell, s), dtype=dt, device="cuda").reshape(-1) for s in (41, 42)]
    e_dev = [plan.energy_potential_async(r) for r in rhos]
    v = torch.empty_like(rhos[0])
    e_dev.append(plan.energy_potential_async(rhos[0], v_out=v))
    torch.cuda.synchronize()
    for r, ed in zip(rhos + rhos[:1], e_dev):
        ref = plan.energy_potential(r)
        got = dict(zip(og.Plan.ENERGY_KEYS, ed.cpu().tolist()))
        for k in og.Plan.ENERGY_KEYS:
            assert abs(got[k] - ref[k]) <= 1e-13 * max(1.0, abs(ref[k])), (k, got[k], ref[k])
    vr = torch.empty_like(v)
    plan.energy_potential(rhos[0], vr)
    assert torch.equal(v, vr)
    plan.close()


def test_module_level_minimize_matches_the_plan():
    cell = fcc_cell(n=16)
    rho, res = og.minimize(cell, tol_F_per_ion=1e-10, tol_residual=1e-7)
    assert res["converged"] and rho.numel() == 16 ** 3
    plan = og.plan_for_cell(cell)
    r2 = torch.empty_like(rho)
    ref = plan.minimize(r2, start_uniform=True, tol_F_per_ion=1e-10, tol_residual=1e-7)
    plan.close()
    assert res["F_total"] == ref["F_total"] and torch.equal(rho, r2)
    # a warm start from the converged density stays there
    rho3, res3 = og.minimize(cell, rho=rho, tol_F_per_ion=1e-10, tol_residual=1e-7)
    assert res3["converged"] and abs(res3["F_total"] - res["F_total"]) < 1e-9


@pytest.mark.parametrize("n,precision", [(8, "fp64"), (512, "fp32"), (512, "fp64")])
def test_grid_size_limits_uniform_density(n, precision):
    # the smallest and largest grids a plan accepts (8^3: a 6-bohr cell of 4
    # ions; 512^3: 64 ions in a 40-bohr cell, 0.078 bohr spacing): a uniform
    # density has the oracle's closed-form energies (vW = NL = H = 0; TF, XC
    # and the local term from nbar alone) and the Ewald energy of the ions
    from oracle.functional import uniform_free_energy
    from oracle.cell import ewald_energy
    from workloads.cells import Cell
    L, n_ion = (6.0, 4) if n == 8 else (40.0, 64)
    rng = np.random.default_rng(SEED_BASE + 71 + n)
    cell = Cell(L=L, n=n, Z=np.ones(n_ion), pos=rng.uniform(0, L, size=(n_ion, 3)), theta=0.8)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    nbar = cell.n_electrons / cell.volume
    rho = torch.full((n ** 3,), nbar, dtype=dt, device="cuda")
    e = plan.energy_potential(rho)
    plan.close()
    ref = uniform_free_energy(cell)
    ref_ion = ewald_energy(np.asarray(cell.Z, float), cell.pos, cell.L)
    tol = 1e-9 if precision == "fp64" else 3e-6
    for key, r in (("F_TF", ref["tf"]), ("E_xc", ref["xc"]), ("E_loc", ref["loc"]), ("E_ion", ref_ion)):
        assert abs(e[key] - r) <= tol * max(1.0, abs(r)), (key, e[key], r)
    for key in ("E_vW", "E_H", "E_NL"):
        assert abs(e[key]) <= tol * max(1.0, abs(ref["tf"])), (key, e[key])
    assert abs(e["N_e"] - cell.n_electrons) <= tol * cell.n_electrons


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_preconditioning_pass_at_128_matches_one_block(precision, monkeypatch):
    # on grids from 112 up the one-field preconditioning pass runs on
    # two-block clusters (half a kz plane per block, columns through
    # distributed shared memory); OFDFT_PREC2=0 runs it on one block per plane
    # (FP32 128^3: identical arithmetic, the same bits) or, where a whole FP64
    # plane does not fit, on the tiled chain (the same minimum)
    cell = config_cell(2)
    dt = torch.float32 if precision == "fp32" else torch.float64
    tol = dict(tol_F_per_ion=1e-10, tol_residual=1e-7) if precision == "fp64" else {}
    out = []
    for env in (None, "0"):
        if env is not None:
            monkeypatch.setenv("OFDFT_PREC2", env)
        plan = og.plan_for_cell(cell, precision=precision)
        rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
        r = plan.minimize(rho, start_uniform=True, **tol)
        plan.close()
        assert r["converged"], r
        out.append((r, rho.double().cpu().numpy()))
    (r1, n1), (r2, n2) = out
    if precision == "fp32":
        assert r1["F_total"] == r2["F_total"] and r1["evaluations"] == r2["evaluations"]
        assert np.array_equal(n1, n2)
    else:
        assert abs(r1["F_total"] - r2["F_total"]) / cell.n_ion < 1e-9
        assert np.linalg.norm(n1 - n2) / np.linalg.norm(n2) < 1e-6


# ------------------------------------------------------------ odd grid sizes
# Odd n: the z passes pack two real rows into one length-n complex transform
# (no Nyquist plane; every kz > 0 carries Hermitian weight 2).  The sizes
# include the batched workload's 75 and 81.
ODD = [(9, lambda: random_cell(SEED_BASE + 61, 2, 1.0, 1.5, 0.8, 9)),
       (15, lambda: random_cell(SEED_BASE + 62, 3, 3.0, 1.4, 0.5, 15)),
       (25, lambda: random_cell(SEED_BASE + 63, 5, 1.0, 2.0, 1.2, 25)),
       (45, lambda: random_cell(SEED_BASE + 64, 9, 4.0, 1.2, 0.3, 45)),
       (75, lambda: random_cell(SEED_BASE + 65, 30, 1.0, 2.2, 1.0, 75)),
       (81, lambda: random_cell(SEED_BASE + 66, 24, 3.0, 1.8, 0.6, 81))]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,mk", ODD)
def test_odd_grids_energy_potential(n, mk, precision):
    cell = mk()
    assert cell.n == n
    rho = rand_density(cell, 6)
    if precision == "fp32":
        rho = rho.astype(np.float32).astype(np.float64)
    e, v = gpu_eval(cell, rho, precision=precision)
    ref_e, ref_v = Functional(cell).evaluate(rho)
    tol_e, tol_v = (1e-9, 1e-8) if precision == "fp64" else (1e-5, 1e-4)
    assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < tol_e
    for k_gpu, k_ref in (("F_TF", "tf"), ("E_vW", "vw"), ("E_NL", "nl"), ("E_H", "hartree"),
                         ("E_loc", "loc"), ("E_xc", "xc"), ("E_ion", "ion")):
        assert abs(e[k_gpu] - ref_e[k_ref]) < tol_e * max(1.0, abs(ref_e[k_ref])) * cell.n_ion, (k_gpu, e[k_gpu], ref_e[k_ref])
    assert np.max(np.abs(v - ref_v)) < tol_v * max(1.0, np.max(np.abs(ref_v)))


@pytest.mark.parametrize("n,mk", [ODD[3], ODD[4]])
def test_odd_grids_tiled_path(n, mk, monkeypatch):
    # the five-pass tiled chain (OFDFT_PLANE=0) on odd grids, FP64
    monkeypatch.setenv("OFDFT_PLANE", "0")
    cell = mk()
    rho = rand_density(cell, 7)
    e, v = gpu_eval(cell, rho)
    ref_e, ref_v = Functional(cell).evaluate(rho)
    assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < 1e-9
    assert np.max(np.abs(v - ref_v)) < 1e-8 * max(1.0, np.max(np.abs(ref_v)))


def test_odd_grid_structure_factor_and_shells():
    cell = ODD[3][1]()
    nh = cell.n // 2 + 1
    plan = og.Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc)
    S = torch.empty((cell.n, cell.n, nh), dtype=torch.complex128, device="cuda")
    plan.structure_factor(cell.pos, S_out=S)
    ref = oracle_sf(cell.pos, cell.n, cell.L)[:, :, :nh]
    assert np.max(np.abs(S.cpu().numpy() - ref)) < 1e-11
    rho = rand_density(cell, 8)
    q, s = plan.sei_shells(torch.tensor(rho, device="cuda"), 60)
    plan.close()
    qr, sr = oracle_sei(rho, cell.pos, cell.L, cell.n_electrons, 60)
    assert np.allclose(q, qr, rtol=1e-14)
    assert np.max(np.abs(s - sr)) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_odd_grid_minimisation_matches_oracle(precision):
    # 9 Z=4 ions at r_s = 1.2, theta = 0.3 on 45^3: the converged minimum of
    # the CUDA path against the oracle's (both from the uniform density; the
    # oracle with its kinetic preconditioner, which does not move the minimum)
    cell = ODD[3][1]()
    F = Functional(cell)
    kF = (3 * math.pi ** 2 * cell.n_electrons / cell.volume) ** (1 / 3)
    ref = lbfgs(F, tol_F=1e-11, tol_R=1e-8, max_iter=3000, precond_c=4 * (0.5 * kF ** 2 + cell.T))
    assert ref.converged
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
    tol = dict(tol_F_per_ion=1e-11, tol_residual=1e-8) if precision == "fp64" else {}
    out = plan.minimize(rho, start_uniform=True, max_iter=3000, **tol)
    plan.close()
    assert out["converged"], out
    n_gpu = rho.double().cpu().numpy().reshape((cell.n,) * 3)
    dF = abs(out["F_total"] - ref.energies["total"]) / cell.n_ion
    dn = np.linalg.norm(n_gpu - ref.rho) / np.linalg.norm(ref.rho)
    print(f"45^3 {precision}: |dF|/ion = {dF:.2e}, rel-L2 density = {dn:.2e}")
    assert dF < 1e-6
    if precision == "fp64":
        assert dn < 1e-5


# ------------------------------------------- density parity, workload extremes
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_128_density_matches_converged_oracle(precision):
    # the oracle's converged 128^3 density (tests/golden, written from oracle/
    # alone, float32) against the GPU minimum: 1e-5 relative L2 in FP64; the
    # FP32-bulk value is printed and bounded
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_density_rand64_H_rs2_n128.npy")
    ref = np.load(path).astype(np.float64).reshape(-1)
    cell = config_cell(2)
    plan = og.plan_for_cell(cell, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
    tol = dict(tol_F_per_ion=1e-9, tol_residual=1e-6) if precision == "fp64" else {}
    out = plan.minimize(rho, start_uniform=True, **tol)
    plan.close()
    assert out["converged"], out
    n = rho.double().cpu().numpy()
    dn = np.linalg.norm(n - ref) / np.linalg.norm(ref)
    print(f"128^3 {precision}: rel-L2 density vs oracle = {dn:.2e}")
    assert dn < (1e-5 if precision == "fp64" else 5e-5)


# cfg 3's ranges at their ends: theta = 0.1 (strongly degenerate) and 2.0,
# Z = 4 at r_s = 1 (the densest cells; r_s < 1 inside the ions, the PZ81
# high-density branch) and Z = 1 at r_s = 3
EXTREMES = [("theta0.1", lambda: random_cell(SEED_BASE + 81, 12, 3.0, 2.0, 0.1, 40)),
            ("theta2.0", lambda: random_cell(SEED_BASE + 82, 12, 1.0, 2.0, 2.0, 40)),
            ("Z4_rs1", lambda: random_cell(SEED_BASE + 83, 16, 4.0, 1.0, 0.5, 48)),
            ("Z1_rs3", lambda: random_cell(SEED_BASE + 84, 10, 1.0, 3.0, 1.0, 48))]


@pytest.mark.parametrize("name,mk", EXTREMES)
def test_minimisation_at_workload_extremes_matches_oracle(name, mk):
    cell = mk()
    F = Functional(cell)
    kF = (3 * math.pi ** 2 * cell.n_electrons / cell.volume) ** (1 / 3)
    ref = lbfgs(F, tol_F=1e-11, tol_R=1e-8, max_iter=4000, precond_c=4 * (0.5 * kF ** 2 + cell.T),
                precond_k=1.0, precond_h=1.5)
    assert ref.converged
    res = {}
    for precision in ("fp64", "fp32"):
        plan = og.plan_for_cell(cell, precision=precision)
        dt = torch.float32 if precision == "fp32" else torch.float64
        rho = torch.empty(cell.n ** 3, dtype=dt, device="cuda")
        tol = dict(tol_F_per_ion=1e-11, tol_residual=1e-8) if precision == "fp64" else {}
        out = plan.minimize(rho, start_uniform=True, max_iter=4000, **tol)
        plan.close()
        assert out["converged"], (precision, out)
        n_gpu = rho.double().cpu().numpy().reshape((cell.n,) * 3)
        res[precision] = (abs(out["F_total"] - ref.energies["total"]) / cell.n_ion,
                          np.linalg.norm(n_gpu - ref.rho) / np.linalg.norm(ref.rho))
    print(f"{name}: fp64 |dF|/ion {res['fp64'][0]:.2e} rel-L2 {res['fp64'][1]:.2e}; "
          f"fp32 |dF|/ion {res['fp32'][0]:.2e} rel-L2 {res['fp32'][1]:.2e}")
    assert res["fp64"][0] < 1e-6 and res["fp64"][1] < 1e-5
    assert res["fp32"][0] < 1e-6


# ------------------------------------------------- FP64 Fermi-Dirac inversion
def test_fp32_plan_with_fp64_fermi_dirac_inversion():
    # TF alone on a density whose y = pi^2 n / (sqrt2 T^1.5) spans e^-30 .. e^22
    # (the classical tail, the fitted range and the degenerate limit), the same
    # FP32-representable values in both plans: with fd64 the FP32 plan's F_TF
    # equals the FP64 plan's to FP64-class accuracy (its inversion is FP64; only
    # the per-point FP32 products and sums remain) and v_TF to FP32 rounding
    cell = random_cell(SEED_BASE + 91, 4, 1.0, 2.0, 0.7, 32)
    T = cell.T
    cy = math.pi ** 2 / (math.sqrt(2.0) * T ** 1.5)
    rng = np.random.default_rng(5)
    logy = rng.uniform(-30.0, 22.0, size=cell.n ** 3)
    rho = (np.exp(logy) / cy).astype(np.float32).astype(np.float64)
    out = {}
    for name, prec, fd64 in (("fp64", "fp64", False), ("fp32_fd64", "fp32", True), ("fp32", "fp32", False)):
        plan = og.plan_for_cell(cell, precision=prec, terms=og.TERM_TF, fd64=fd64)
        dt = torch.float32 if prec == "fp32" else torch.float64
        r = torch.tensor(rho, dtype=dt, device="cuda")
        v = torch.empty_like(r)
        e = plan.energy_potential(r, v)
        plan.close()
        out[name] = (e["F_TF"], v.double().cpu().numpy())
    F64, v64 = out["fp64"]
    # v_TF = T eta: error of eta relative to max(|eta|, 1) (eta crosses 0)
    err = {k: (abs(out[k][0] - F64) / abs(F64),
               float(np.max(np.abs(out[k][1] - v64) / np.maximum(np.abs(v64), T))))
           for k in ("fp32_fd64", "fp32")}
    print("F_TF rel err, max v_TF err / max(|v|, T):", err)
    # (the remaining F_TF error, 1.6e-9 measured, is the FP32 sums of the
    # per-point values; the FP32 fit's inversion leaves 4e-7)
    assert err["fp32_fd64"][0] < 3e-9
    assert err["fp32_fd64"][1] < 1.2e-7            # one FP32 rounding of T eta
    # the FP32 fit over the same range: 4e-7 in F_TF, 2.8e-6 in eta (measured)
    assert err["fp32"][0] < 1e-6 and err["fp32"][1] < 1e-5


def test_register_passes_at_256_match_the_generic_ones(monkeypatch):
    # 256^3 FP32 runs its z passes with register transforms (k_zfwd256,
    # k_zinv256) and its x-y transforms with the G-space terms in the
    # eight-block cluster plane pass (k_plane256cl, plane layout).
    # OFDFT_P256=0 selects the register y and x/G-space passes on the tiled
    # layout instead (k_ypass256, k_xgspace256), OFDFT_Z256=0 the generic
    # shared-memory passes.  The tiled register passes keep the generic
    # passes' butterflies, twiddles, their order and the per-thread grouping
    # of the G-space sums: the same potential bits, energies equal up to the
    # rounding of the compensated block sums.  The plane pass splits the x
    # transforms as 32 x 8 instead of 16 x 16 and sums other runs of FP32
    # terms per thread: FP32 rounding
    # Every row block the autotuner may pick (8, 16 or 32 rows per z block)
    # is checked: the z passes' team buffers and the plane-layout split
    # depend on it.
    cell = config_cell(4)
    nbar = cell.n_electrons / cell.volume
    rng = np.random.default_rng(9)
    rho = torch.tensor(nbar * (1 + 0.3 * rng.random(cell.n ** 3)), dtype=torch.float32, device="cuda")
    cases = [({"OFDFT_ZR": zr}, zr == "16") for zr in ("8", "16", "32")]
    cases += [({"OFDFT_P256": "0", "OFDFT_ZR": zr}, zr == "16") for zr in ("8", "16", "32")]
    cases += [({"OFDFT_Z256": "0"}, True)]
    out = []
    for env, with_min in cases:
        for k in ("OFDFT_P256", "OFDFT_Z256", "OFDFT_ZR"):
            monkeypatch.delenv(k, raising=False)
        for k, val in env.items():
            monkeypatch.setenv(k, val)
        plan = og.plan_for_cell(cell, precision="fp32")
        v = torch.empty_like(rho)
        e = plan.energy_potential(rho, v)
        m = None
        if with_min:
            r2 = torch.empty_like(rho)
            m = plan.minimize(r2, start_uniform=True)
            assert m["converged"], (env, m)
            m = (m["F_total"], r2.double().cpu().numpy())
        plan.close()
        out.append((e, v.cpu(), m))
    e2, v2, (f2, n2) = out[-1]
    for (env, _), (e1, v1, m1) in zip(cases, out[:-1]):
        if "OFDFT_P256" in env:
            assert torch.equal(v1, v2), env
            # other row blocks: other runs of FP32 terms in the per-thread
            # real-space sums
            tol = 1e-12 if env["OFDFT_ZR"] == "8" else 1e-9
        else:
            assert ((v1 - v2).abs().max() / v2.abs().max()).item() < 2e-6, env
            tol = 5e-7
        # F_total is a difference of terms of ~1e3 Ha: it is held to the
        # terms' scale
        scale = sum(abs(e2[k]) for k in ("F_TF", "E_vW", "E_NL", "E_H", "E_loc", "E_xc", "E_ion"))
        for k in e1:
            ref = scale if k == "F_total" else max(1.0, abs(e2[k]))
            assert abs(e1[k] - e2[k]) <= tol * ref, (env, k, e1[k], e2[k])
        if m1 is not None:
            # the minimisations see energies that differ in the last bits, so
            # their paths part; both end inside the convergence tolerance of
            # the same minimum
            f1, n1 = m1
            assert abs(f1 - f2) / cell.n_ion < 1e-6, env
            assert np.linalg.norm(n1 - n2) / np.linalg.norm(n2) < 5e-5, env


def test_256_passes_with_three_fields(monkeypatch):
    # a = 5/6: n^a is a third transformed field beside n and psi, so the
    # 256^3 z passes take 48 row transforms per 16-row block (two rounds of
    # their 32 teams) and the cluster plane pass three fields per launch.
    # The three forms against each other (the register passes bit for bit
    # with the generic ones) and against the oracle; 16 Z=3 ions, a smooth
    # density of a few low-frequency modes.
    n = 256
    cell = random_cell(11, 16, 3.0, 2.5, 0.3, n)
    nbar = cell.n_electrons / cell.volume
    rng = np.random.default_rng(5)
    x = np.arange(n) * (2 * np.pi / n)
    X, Y, Zc = np.meshgrid(x, x, x, indexing="ij")
    pert = np.zeros((n, n, n))
    for _ in range(6):
        m = rng.integers(-3, 4, size=3)
        pert += rng.uniform(0.02, 0.05) * np.cos(m[0] * X + m[1] * Y + m[2] * Zc + rng.uniform(0, 2 * np.pi))
    rho = nbar * (1.0 + pert)
    rho *= cell.n_electrons / (rho.sum() * cell.volume / rho.size)
    out = []
    envs = ({}, {"OFDFT_P256": "0"}, {"OFDFT_Z256": "0"})
    for env in envs:
        for k in ("OFDFT_P256", "OFDFT_Z256"):
            monkeypatch.delenv(k, raising=False)
        for k, val in env.items():
            monkeypatch.setenv(k, val)
        out.append(gpu_eval(cell, rho.reshape(-1), precision="fp32", alpha=5 / 6))
    (e1, v1), (e2, v2), (e3, v3) = out
    assert np.array_equal(v2, v3)
    # the n^a field keeps its mean (the psi field's is removed before its
    # transform), so each form's FP32 rounding scales with that mean, and the
    # two groupings of the x transform differ by more than in the two-field
    # case (2.8e-6 of max|v| measured)
    assert np.max(np.abs(v1 - v3)) / np.max(np.abs(v3)) < 1e-5
    ref_e, ref_v = Functional(cell, alpha=5 / 6).evaluate(rho)
    for e, v in ((e1, v1), (e3, v3)):
        err_v = np.max(np.abs(v.reshape(n, n, n) - ref_v)) / np.max(np.abs(ref_v))
        print("three fields: |dF|/ion", abs(e["F_total"] - ref_e["total"]) / cell.n_ion, "max|dv|/max|v|", err_v)
        assert abs(e["F_total"] - ref_e["total"]) / cell.n_ion < 1e-6
        assert abs(e["E_NL"] - ref_e["nl"]) / cell.n_ion < 1e-6
        assert err_v < 5e-4

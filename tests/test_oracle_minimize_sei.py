"""Pins of the oracle minimiser (properties of the variational minimum) and of
the electron-ion structure factor (Methods, S_ab(q) definition)."""
import math

import numpy as np
import pytest

from oracle.functional import Functional
from oracle.minimize import lbfgs
from oracle.sei import sei_shells
from oracle.cell import structure_factor
from workloads import fcc_cell, random_cell


@pytest.fixture(scope="module")
def small_min():
    c = fcc_cell(n=16)
    F = Functional(c)
    r = lbfgs(F, tol_F=1e-11, tol_R=1e-8, max_iter=400)
    return c, F, r


def test_minimum_conserves_electrons_and_is_stationary(small_min):
    c, F, r = small_min
    assert r.converged
    assert abs(F.dV * r.rho.sum() - c.n_electrons) < 1e-12 * c.n_electrons
    assert r.energies["residual"] < 1e-8


def test_minimum_is_lower_than_perturbations(small_min):
    c, F, r = small_min
    rng = np.random.default_rng(2)
    for _ in range(3):
        p = r.psi * (1 + 1e-3 * rng.standard_normal(r.psi.shape))
        assert F.evaluate_psi(p)[0]["total"] > r.energies["total"]


def test_minimum_independent_of_optimizer_constants(small_min):
    c, F0, r0 = small_min
    F = Functional(c)
    rng = np.random.default_rng(9)
    start = np.sqrt(c.n_electrons / c.volume) * (1 + 0.05 * rng.standard_normal((16,) * 3))
    r = lbfgs(F, psi0=start, m=4, c2=0.5, tol_F=1e-11, tol_R=1e-8, max_iter=600)
    assert r.converged
    assert abs(r.energies["total"] - r0.energies["total"]) / c.n_ion < 1e-10
    assert np.linalg.norm(r.rho - r0.rho) / np.linalg.norm(r0.rho) < 1e-6


def test_preconditioned_minimiser_reaches_the_same_minimum(small_min):
    # H0 = gamma P with the kinetic preconditioner P changes the path, not the
    # minimum; on this cell it also needs fewer iterations
    c, F0, r0 = small_min
    F = Functional(c)
    kF = (3 * math.pi ** 2 * c.n_electrons / c.volume) ** (1 / 3)
    r = lbfgs(F, precond_c=0.5 * kF ** 2, tol_F=1e-11, tol_R=1e-8, max_iter=400)
    assert r.converged
    assert abs(r.energies["total"] - r0.energies["total"]) / c.n_ion < 1e-10
    assert np.linalg.norm(r.rho - r0.rho) / np.linalg.norm(r0.rho) < 1e-6
    assert r.iterations < r0.iterations


def test_hartree_and_kernel_preconditioner_reaches_the_same_minimum(small_min):
    # the preconditioner with the kernel's curvature and the Hartree term
    # 8 pi nbar / G^2 is another symmetric positive-definite H0: same minimum
    c, F0, r0 = small_min
    F = Functional(c)
    kF = (3 * math.pi ** 2 * c.n_electrons / c.volume) ** (1 / 3)
    r = lbfgs(F, precond_c=4 * (0.5 * kF ** 2 + c.T), precond_k=1.0, precond_h=1.5, tol_F=1e-11,
              tol_R=1e-8, max_iter=400)
    assert r.converged
    assert abs(r.energies["total"] - r0.energies["total"]) / c.n_ion < 1e-10
    assert np.linalg.norm(r.rho - r0.rho) / np.linalg.norm(r0.rho) < 1e-6


def test_sei_uniform_is_zero():
    c = random_cell(21, 8, 1.0, 1.5, 1.0, 16)
    q, s = sei_shells(np.full((16,) * 3, c.n_electrons / c.volume), c.pos, c.L, c.n_electrons, 40)
    assert np.max(np.abs(s)) < 1e-12
    assert np.all(np.diff(q) > 0)


def test_sei_of_gaussian_density_closed_form():
    # n = sum_I Z g_s(r - R_I): n_e(G) = Z exp(-G^2 s^2/2) S(G), so
    # S_ei(G) = Z exp(-G^2 s^2 / 2) |S(G)|^2 / sqrt(N_e N_i) (shell-averaged)
    L, n, s, Z = 9.0, 48, 0.5, 1.0
    pos = np.array([[1.0, 2.0, 3.0], [5.0, 5.5, 1.5], [7.5, 3.0, 7.0]])
    x = np.arange(n) * L / n
    X, Y, Zc = np.meshgrid(x, x, x, indexing="ij")
    rho = np.zeros((n, n, n))
    for p in pos:
        d2 = 0
        for ax, comp in zip((X, Y, Zc), p):
            d = ax - comp
            d -= L * np.round(d / L)
            d2 = d2 + d * d
        rho += Z * np.exp(-d2 / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    ne = Z * len(pos)
    q, got = sei_shells(rho, pos, L, ne, 30)
    S = structure_factor(pos, n, L)
    m = np.fft.fftfreq(n) * n
    m2 = (m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2).round().astype(int)
    G2 = (2 * math.pi / L) ** 2 * m2
    ref_grid = Z * np.exp(-G2 * s * s / 2) * np.abs(S) ** 2 / math.sqrt(ne * len(pos))
    vals = np.unique(m2[m2 > 0])[:30]
    ref = np.array([ref_grid[m2 == v].mean() for v in vals])
    assert np.allclose(got, ref, atol=1e-9)


def test_sii_single_ion_is_one():
    from oracle.sei import sii_shells
    q, s = sii_shells(np.array([[0.3, 1.7, 2.2]]), 5.0, 16, 40)
    assert np.allclose(s, 1.0, rtol=0, atol=1e-13)


def test_sii_simple_cubic_lattice_counts_reciprocal_vectors():
    # M^3 ions on a simple cubic lattice in the cell: S(G) = N_i when every
    # component of m is a multiple of M, else 0, so S_ii(shell) = N_i x (share
    # of the shell's grid vectors that are multiples of M), counted by brute force
    from oracle.sei import sii_shells
    M, n, L = 3, 18, 7.0
    g = np.arange(M) * L / M
    pos = np.array([[x, y, z] for x in g for y in g for z in g]) + 0.4
    q, s = sii_shells(pos, L, n, 60)
    ms = [m if m < n // 2 else m - n for m in range(n)]
    count, hit = {}, {}
    for a in ms:
        for b in ms:
            for c in ms:
                k = a * a + b * b + c * c
                if k == 0:
                    continue
                count[k] = count.get(k, 0) + 1
                hit[k] = hit.get(k, 0) + (a % M == 0 and b % M == 0 and c % M == 0)
    keys = sorted(count)[:60]
    ref = np.array([M ** 3 * hit[k] / count[k] for k in keys])
    assert np.allclose(q, 2 * math.pi / L * np.sqrt(keys), rtol=1e-15)
    assert np.allclose(s, ref, atol=1e-10)


def test_sei_direct_equals_full_grid_form():
    from oracle.sei import sei_shells_direct
    c = random_cell(23, 11, 1.0, 1.7, 1.0, 20)
    rng = np.random.default_rng(4)
    rho = c.n_electrons / c.volume * (1 + 0.2 * rng.random((20,) * 3))
    q1, s1 = sei_shells(rho, c.pos, c.L, c.n_electrons, 50)
    q2, s2 = sei_shells_direct(rho, c.pos, c.L, c.n_electrons, 50)
    assert np.allclose(q1, q2, rtol=1e-15)
    assert np.abs(s1 - s2).max() < 1e-12 * max(1.0, np.abs(s1).max())

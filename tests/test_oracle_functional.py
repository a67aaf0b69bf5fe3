"""Pins of the oracle functional F[n] (Eq. 1 terms plus Hartree, local PP, XC)
against closed forms, brute force and the response condition of Eq. 2."""
import itertools
import math

import numpy as np
import pytest

from oracle.functional import Functional, fft3, ifft3, uniform_free_energy
from oracle.cell import ewald_energy
from oracle.lindhard import chi0, mean_density_params
from workloads import fcc_cell, random_cell


def test_fft_convention_matches_naive_dft():
    # f~(G) = (1/N) sum_r f(r) exp(-i G.r) on a 6^3 grid, brute force
    rng = np.random.default_rng(1)
    n = 6
    f = rng.standard_normal((n, n, n))
    F = fft3(f)
    m = np.fft.fftfreq(n) * n
    for (a, b, c) in [(0, 0, 0), (1, 2, 3), (5, 0, 4), (3, 3, 3)]:
        s = 0j
        for i, j, k in itertools.product(range(n), repeat=3):
            s += f[i, j, k] * np.exp(-2j * math.pi * (m[a] * i + m[b] * j + m[c] * k) / n)
        assert abs(F[a, b, c] - s / n ** 3) < 1e-13
    assert np.allclose(ifft3(F), f, atol=1e-13)


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 9])
def test_fft_every_entry_against_brute_force_dft(n):
    # every G of an n^3 grid (odd and even n): the O(N^2) sum written out
    # over all r at once, with the 1/N of the forward convention
    rng = np.random.default_rng(100 + n)
    f = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    r = np.array(list(itertools.product(range(n), repeat=3)), dtype=float)       # [N, 3]
    m = np.array(list(itertools.product(range(n), repeat=3)), dtype=float)       # [N, 3]
    phase = np.exp(-2j * math.pi * (m @ r.T) / n)                                 # [N_G, N_r]
    ref = (phase @ f.reshape(-1)).reshape(n, n, n) / n ** 3
    F = fft3(f)
    assert np.max(np.abs(F - ref)) < 1e-14 * max(1.0, np.max(np.abs(ref))) * n ** 2
    # Parseval with this normalisation: sum_r |f|^2 = N sum_G |f~|^2
    assert abs(np.sum(np.abs(f) ** 2) - n ** 3 * np.sum(np.abs(F) ** 2)) < 1e-11 * np.sum(np.abs(f) ** 2)
    # the inverse returns the real field: round trip of the real part
    assert np.max(np.abs(ifft3(fft3(f.real)) - f.real)) < 1e-13


@pytest.mark.parametrize("n", [5, 8, 9])
def test_fft_single_plane_wave_is_a_delta(n):
    # f(r) = exp(i G0.r) with G0 = (2 pi / L) m0 has f~ = 1 at m0 and 0 elsewhere
    m0 = (1, n - 2, 3 % n)
    x = np.arange(n)
    f = np.exp(2j * math.pi * (m0[0] * x[:, None, None] + m0[1] * x[None, :, None] + m0[2] * x[None, None, :]) / n)
    F = fft3(f)
    expect = np.zeros((n, n, n), dtype=complex)
    expect[m0] = 1.0
    assert np.max(np.abs(F - expect)) < 1e-14


def test_uniform_density_closed_form():
    c = fcc_cell()
    F = Functional(c)
    e, v = F.evaluate(np.full((c.n,) * 3, c.n_electrons / c.volume))
    ref = uniform_free_energy(c)
    assert abs(ref["tf"] - 0.32317493429316) < 1e-11
    for k in ("tf", "xc", "loc"):
        assert abs(e[k] - ref[k]) < 1e-11 * max(1, abs(ref[k])), k
    for k in ("vw", "nl", "hartree"):
        assert abs(e[k]) < 1e-12, k


def _cos_field(n, L, m, base, amp):
    x = np.arange(n) * L / n
    G0 = 2 * math.pi / L * m
    return base + amp * np.cos(G0 * x)[:, None, None] * np.ones((n, n, n)), G0


def test_vw_cosine_closed_form():
    # phi = a + b cos(G0 x): E_vW = Omega b^2 G0^2 / 4
    c = random_cell(2, 4, 1.0, 1.5, 1.0, 16)
    F = Functional(c, terms=("vw",))
    phi, G0 = _cos_field(16, c.L, 3, 0.2, 0.05)
    e, _ = F.evaluate(phi ** 2)
    assert abs(e["vw"] - c.volume * 0.05 ** 2 * G0 ** 2 / 4) < 1e-12


def test_hartree_cosine_closed_form():
    # n = nbar + A cos(G0 x): E_H = pi Omega A^2 / G0^2
    c = random_cell(2, 4, 1.0, 1.5, 1.0, 16)
    F = Functional(c, terms=("hartree",))
    rho, G0 = _cos_field(16, c.L, 2, 0.03, 0.01)
    e, _ = F.evaluate(rho)
    assert abs(e["hartree"] - math.pi * c.volume * 0.01 ** 2 / G0 ** 2) < 1e-13


def test_hartree_of_gaussians_matches_ewald():
    # well separated Gaussian charges Q_I with density Q g_s(r - R_I), g_s the
    # normalised Gaussian of standard deviation s (transform exp(-G^2 s^2/2)):
    # E_H(G != 0) is the Ewald reciprocal sum at eta = 1/(2s), so
    # E_H = E_Ewald(point) + sum Q^2 / (2 sqrt(pi) s) + 2 pi s^2 (sum Q)^2 / Omega
    # (self and background terms at that eta; the real-space erfc part is
    # below 1e-20 at these separations)
    L, n, s = 10.0, 64, 0.45
    pos = np.array([[2.0, 2.5, 3.0], [7.0, 6.5, 5.5]])
    Q = np.array([1.0, 2.0])
    x = np.arange(n) * L / n
    X, Y, Zc = np.meshgrid(x, x, x, indexing="ij")
    rho = np.zeros((n, n, n))
    for q, p in zip(Q, pos):
        d2 = 0
        for ax, comp in zip((X, Y, Zc), p):
            d = ax - comp
            d -= L * np.round(d / L)
            d2 = d2 + d * d
        rho += q * np.exp(-d2 / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5

    class C:
        pass
    c = C()
    c.n, c.L, c.Z, c.pos, c.T, c.rc = n, L, Q, pos, 1.0, 1.0
    F = Functional(c, terms=("hartree",))
    e, _ = F.evaluate(rho)
    ref = ewald_energy(Q, pos, L) + np.sum(Q ** 2) / (2 * math.sqrt(math.pi) * s) \
        + 2 * math.pi * s * s * np.sum(Q) ** 2 / L ** 3
    assert abs(e["hartree"] - ref) < 1e-6 * abs(ref)


@pytest.mark.parametrize("m", [1, 3, 6])
def test_linear_response_of_noninteracting_part(m):
    # F_s[nbar + eps cos] - F_s[nbar] = (Omega/4) eps^2 (-1/chi0(G0;T)) + O(eps^3)
    c = fcc_cell(n=16)
    F = Functional(c, terms=("tf", "vw", "nl"))
    nbar = c.n_electrons / c.volume
    base = F.evaluate(np.full((16,) * 3, nbar))[0]["total"]
    eps = 1e-4 * nbar
    rho, G0 = _cos_field(16, c.L, m, nbar, eps)
    de = F.evaluate(rho)[0]["total"] - base
    _, mu0, _ = mean_density_params(nbar, c.T)
    pred = c.volume / 4 * eps ** 2 * (-1 / chi0(G0, mu0, c.T))
    assert abs(de / pred - 1) < 5e-6


@pytest.mark.parametrize("terms", [("tf",), ("vw",), ("nl",), ("xc",), ("hartree",), ("loc",),
                                   ("tf", "vw", "nl", "xc", "hartree", "loc")])
def test_potential_is_functional_derivative(terms):
    # [F(n + h dn) - F(n - h dn)] / 2h = dV sum v dn for a random mass-conserving dn
    c = random_cell(4, 6, 3.0, 1.6, 0.7, 16)
    F = Functional(c, terms=terms)
    rng = np.random.default_rng(3)
    nbar = c.n_electrons / c.volume
    rho = nbar * np.exp(0.4 * rng.standard_normal((16,) * 3))
    dn = rng.standard_normal((16,) * 3) * nbar
    dn -= dn.mean()
    h = 1e-5
    ep = F.evaluate(rho + h * dn)[0]["total"]
    em = F.evaluate(rho - h * dn)[0]["total"]
    _, v = F.evaluate(rho)
    lhs = (ep - em) / (2 * h)
    rhs = F.dV * np.sum(v * dn)
    assert abs(lhs - rhs) < 1e-8 * max(1.0, abs(rhs)), (lhs, rhs)


def test_psi_gradient_matches_finite_difference():
    c = random_cell(8, 5, 1.0, 1.7, 1.0, 12)
    F = Functional(c)
    rng = np.random.default_rng(5)
    psi = 1 + 0.2 * rng.standard_normal((12,) * 3)
    dpsi = rng.standard_normal((12,) * 3)
    h = 1e-6
    ep = F.evaluate_psi(psi + h * dpsi)[0]["total"]
    em = F.evaluate_psi(psi - h * dpsi)[0]["total"]
    _, g, _ = F.evaluate_psi(psi)
    assert abs((ep - em) / (2 * h) - F.dV * np.sum(g * dpsi)) < 1e-7 * max(1, abs(ep - em) / (2 * h))
    # scale invariance: g is orthogonal to psi
    assert abs(F.dV * np.sum(g * psi)) < 1e-10 * F.dV * np.sum(np.abs(g * psi))


def test_uniform_nl_energy_is_zero_for_any_alpha():
    c = fcc_cell(n=16)
    for a in (0.5, 5 / 6):
        F = Functional(c, terms=("nl",), alpha=a)
        e, _ = F.evaluate(np.full((16,) * 3, c.n_electrons / c.volume))
        assert abs(e["nl"]) < 1e-12

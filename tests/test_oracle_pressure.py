"""Pins of the oracle's electronic pressure (oracle/pressure.py).

Each term's virial formula is checked against central differences of that
same term's energy, recomputed by the oracle functional on a dilated cell
(L, R_I -> lambda L, lambda R_I; n -> n / lambda^3 on the same grid; the same
temperature), so a dropped factor or a wrong degree in any term fails its own
check.  The uniform Thomas-Fermi gas is pinned to the ideal Fermi gas
pressure (2/3) x kinetic energy density, from Fermi-Dirac integrals done by
direct quadrature here."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle.functional import Functional
from oracle.pressure import pressure
from workloads import random_cell
from workloads.cells import Cell

TERM_KEYS = ("tf", "vw", "nl", "hartree", "loc", "xc", "ion")


def _dilated(cell, lam):
    # same T: T_F scales as lambda^-2, so theta scales as lambda^2
    c = Cell(L=cell.L * lam, n=cell.n, Z=cell.Z, pos=np.asarray(cell.pos) * lam,
             theta=cell.theta * lam * lam, rc=cell.rc, label=cell.label)
    assert abs(c.T - cell.T) < 1e-13 * cell.T
    return c


def _density(cell, seed):
    rng = np.random.default_rng(seed)
    n = cell.n
    x = np.arange(n) / n
    sm = sum(rng.uniform(0.2, 1.0) * np.cos(2 * math.pi * (k[0] * x[:, None, None] + k[1] * x[None, :, None]
                                                               + k[2] * x[None, None, :]) + rng.uniform(0, 6.28))
             for k in rng.integers(-2, 3, size=(4, 3)))
    rho = np.exp(0.3 * sm / 3.0)
    return rho * cell.n_electrons / (rho.sum() * cell.volume / rho.size)


def _fd_pressure(cell, rho, alpha, h):
    """-(1/(3 Omega)) dE_term/dlambda by Richardson-extrapolated central differences."""
    def energies(lam):
        F = Functional(_dilated(cell, lam), alpha=alpha)
        return F.evaluate(rho / lam ** 3)[0]

    def central(s):
        ep, em = energies(1 + s), energies(1 - s)
        return {k: (ep[k] - em[k]) / (2 * s) for k in TERM_KEYS}

    d1, d2 = central(h), central(h / 2)
    Om = cell.volume
    return {k: -((4 * d2[k] - d1[k]) / 3) / (3 * Om) for k in TERM_KEYS}


@pytest.mark.parametrize("alpha", [0.5, 5.0 / 6.0])
def test_pressure_terms_match_energy_differences(alpha):
    cell = random_cell(41, 4, 1.0, 1.6, 0.8, 12)
    rho = _density(cell, 7)
    p = pressure(cell, rho, alpha=alpha)
    ref = _fd_pressure(cell, rho, alpha, 2e-3)
    scale = max(abs(v) for v in ref.values())
    for k in TERM_KEYS:
        assert abs(p[k] - ref[k]) < 1e-7 * scale, (k, p[k], ref[k])
    assert abs(p["total"] - sum(ref.values())) < 1e-7 * scale


def test_uniform_tf_pressure_is_the_ideal_fermi_gas():
    # P = (2/3) tau, tau = sqrt2/pi^2 T^(5/2) F_{3/2}(eta), n = sqrt2/pi^2 T^(3/2) F_{1/2}(eta)
    cell = random_cell(42, 3, 1.0, 2.0, 0.7, 8)
    nbar = cell.n_electrons / cell.volume
    T = cell.T

    def F(j, eta):
        return integrate.quad(lambda x: x ** j / (1.0 + math.exp(min(x - eta, 700.0))), 0, max(eta, 0) + 60,
                              epsabs=0, epsrel=1e-13, limit=200)[0]

    c = math.sqrt(2.0) / math.pi ** 2
    eta = optimize.brentq(lambda e: c * T ** 1.5 * F(0.5, e) - nbar, -30, 60, xtol=1e-15, rtol=1e-15)
    expect = 2.0 / 3.0 * c * T ** 2.5 * F(1.5, eta)
    p = pressure(cell, np.full((8,) * 3, nbar), terms=("tf",))
    assert abs(p["tf"] - expect) < 1e-10 * expect
    assert p["total"] == pytest.approx(p["tf"] + p["ion"], rel=1e-15)


def test_uniform_density_has_no_gradient_or_hartree_pressure():
    cell = random_cell(43, 3, 1.0, 2.0, 0.7, 8)
    nbar = cell.n_electrons / cell.volume
    p = pressure(cell, np.full((8,) * 3, nbar))
    assert abs(p["vw"]) < 1e-14 and abs(p["hartree"]) < 1e-14 and abs(p["nl"]) < 1e-12
    # local term of a uniform density: only G = 0 survives, (1/3) n~(0) V(0) 3
    assert p["loc"] == pytest.approx(nbar * math.pi * cell.rc ** 2 * cell.n_electrons / cell.volume, rel=1e-12)

"""Pins of the oracle's Fermi-Dirac integrals and finite-T Thomas-Fermi term
(F_s^TF of Eq. 1) against closed forms, limits and an independent library."""
import math
import os

import numpy as np
import pytest
from scipy.special import zeta, gamma

from oracle import fermi_dirac as fd

HERE = os.path.dirname(__file__)


def golden():
    rows = []
    with open(os.path.join(HERE, "golden", "fd_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                nu, eta, val = line.split()
                rows.append((float(nu), float(eta), float(val)))
    return rows


def test_golden_polylog_values():
    for nu, eta, val in golden():
        got = float(fd.fd_integral(nu, np.array([eta]))[0])
        assert abs(got - val) <= 1e-13 * abs(val), (nu, eta, got, val)


@pytest.mark.parametrize("nu", [-0.5, 0.5, 1.5])
def test_closed_form_at_zero(nu):
    # I_nu(0) = Gamma(nu+1) (1 - 2^-nu) zeta(nu+1)
    ref = gamma(nu + 1) * (1 - 2.0 ** (-nu)) * zeta(nu + 1)
    got = float(fd.fd_integral(nu, np.array([0.0]))[0])
    assert abs(got - ref) < 1e-14 * abs(ref)


def test_against_mpmath_polylog_grid():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    etas = np.array([-30.0, -7.3, -1.1, 0.3, 2.2, 9.7, 27.0, 61.0])
    im, ih, i3 = fd.fd_integrals(etas)
    for k, eta in enumerate(etas):
        for nu, got in ((-0.5, im[k]), (0.5, ih[k]), (1.5, i3[k])):
            ref = float(-mp.gamma(nu + 1) * mp.re(mp.polylog(nu + 1, -mp.exp(eta))))
            assert abs(got - ref) <= 2e-14 * abs(ref), (nu, eta, got, ref)


def test_boltzmann_limit():
    eta = np.array([-40.0, -35.0])
    for nu in (-0.5, 0.5, 1.5):
        got = fd.fd_integral(nu, eta)
        ref = gamma(nu + 1) * np.exp(eta)
        assert np.allclose(got, ref, rtol=1e-14)


def test_sommerfeld_limit():
    eta = np.array([400.0, 900.0])
    for nu in (0.5, 1.5):
        got = fd.fd_integral(nu, eta)
        ref = eta ** (nu + 1) / (nu + 1) * (1 + math.pi ** 2 * nu * (nu + 1) / (6 * eta ** 2))
        assert np.allclose(got, ref, rtol=1e-10)


def test_derivative_identity():
    # d I_nu / d eta = nu I_{nu-1}
    eta = np.array([-3.0, 0.7, 4.5, 20.0])
    h = 1e-4
    for nu, lower in ((1.5, 0.5), (0.5, -0.5)):
        fd_ = (fd.fd_integral(nu, eta + h) - fd.fd_integral(nu, eta - h)) / (2 * h)
        assert np.allclose(fd_, nu * fd.fd_integral(lower, eta), rtol=1e-8)


def test_inverse_round_trip():
    eta = np.linspace(-40, 200, 241)
    y = fd.fd_integral(0.5, eta)
    back = fd.inverse_fd_half(y)
    assert np.max(np.abs(back - eta) / np.maximum(1, np.abs(eta))) < 1e-13


def test_uniform_tf_fcc_cell():
    # 4-ion fcc, Z = 3, a = 7.6 bohr, theta = 0.5 (mpmath values)
    Omega = 7.6 ** 3
    nbar = 12 / Omega
    T = 0.5 * 0.5 * (3 * math.pi ** 2 * nbar) ** (2 / 3)
    assert abs(nbar - 0.027336346406182) < 1e-14
    assert abs(T - 0.21712724482783) < 1e-13
    f, v, eta = fd.tf_free_energy_density(np.array([nbar]), T)
    assert abs(eta[0] - 1.4862241685178) < 1e-12
    assert abs(v[0] - 0.32269975890680) < 1e-12
    assert abs(f[0] - 7.3620182946941e-4) < 1e-16
    assert abs(Omega * f[0] - 0.32317493429316) < 1e-12


def test_uniform_tf_other_cells():
    # H at r_s = 2, theta = 1, 64 e-; Z = 3 at r_s = 2.5, theta = 0.3, 3072 e-
    for ne, rs, theta, T_ref, eta_ref, F_ref in (
            (64, 2.0, 1.0, 0.46039606904411, -0.021460754986923, -33.962359446165),
            (3072, 2.5, 0.3, 0.088396045256469, 3.0486076717427, 352.79912055175)):
        Omega = ne * 4 * math.pi * rs ** 3 / 3
        nbar = ne / Omega
        T = theta * 0.5 * (3 * math.pi ** 2 * nbar) ** (2 / 3)
        assert abs(T - T_ref) < 1e-12
        f, v, eta = fd.tf_free_energy_density(np.array([nbar]), T)
        assert abs(eta[0] - eta_ref) < 1e-11
        assert abs(Omega * f[0] - F_ref) < 1e-9 * abs(F_ref)


def test_zero_temperature_limit():
    # T -> 0: f -> (3/10)(3 pi^2)^(2/3) n^(5/3)
    n = 0.027336346406182
    f, v, _ = fd.tf_free_energy_density(np.array([n]), 1e-5)
    ref = 0.3 * (3 * math.pi ** 2) ** (2 / 3) * n ** (5 / 3)
    assert abs(ref - 7.1225586946e-3) < 1e-12
    assert abs(f[0] - ref) < 1e-6 * ref


def test_thermodynamic_consistency():
    # d f / d n = mu = T eta
    n = np.array([1e-4, 0.0273, 0.5, 3.0])
    T = 0.3
    h = 1e-6 * n
    fp, _, _ = fd.tf_free_energy_density(n + h, T)
    fm, _, _ = fd.tf_free_energy_density(n - h, T)
    _, v, _ = fd.tf_free_energy_density(n, T)
    assert np.allclose((fp - fm) / (2 * h), v, rtol=1e-7)


def test_golden_file_is_what_its_generator_writes():
    # the stored values come from tests/golden/make_fd_values.py (mpmath only)
    pytest.importorskip("mpmath")
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_fd_values", os.path.join(HERE, "golden", "make_fd_values.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    stored = golden()
    fresh = mod.values()
    assert len(stored) == len(fresh)
    for (nu, eta, val), (nu2, eta2, v2) in zip(stored, fresh):
        assert (nu, eta) == (nu2, eta2) and val == float(v2)

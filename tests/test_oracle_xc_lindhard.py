"""Pins of the PZ LDA (Methods) and of the finite-T Lindhard response that
fixes the F_0^NL kernel (Eq. 2)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import xc
from oracle.lindhard import chi0, chi0_zero_T, mean_density_params, kernel_value, ALPHA
from oracle import fermi_dirac as fd


def test_exchange_closed_form():
    n = np.array([1e-3, 0.0273, 1.0, 10.0])
    ex, vx = xc.exchange(n)
    rs = (3 / (4 * math.pi * n)) ** (1 / 3)
    # e_x = -(3/4)(9/(4 pi^2))^(1/3) / r_s = -0.458165293... / r_s
    assert np.allclose(ex, -0.4581652932831429 / rs, rtol=1e-14)
    assert np.allclose(vx, 4 / 3 * ex, rtol=1e-15)


def test_pz_branches_join_smoothly_at_rs_1():
    # e_c and v_c (hence d e_c / d r_s) continuous at r_s = 1, and B, D the
    # printed PZ81 values up to their last printed digit
    n1 = 3 / (4 * math.pi)
    e_lo, v_lo = xc.correlation(np.array([n1 * (1 + 1e-12)]))
    e_hi, v_hi = xc.correlation(np.array([n1 * (1 - 1e-12)]))
    assert abs(e_lo[0] - e_hi[0]) < 1e-13
    assert abs(v_lo[0] - v_hi[0]) < 1e-11
    assert abs(e_hi[0] - (-0.1423 / (1 + 1.0529 + 0.3334))) < 1e-9
    assert abs(xc.B - (-0.048)) < 5e-5 and abs(xc.D - (-0.0116)) < 5e-5


@pytest.mark.parametrize("n0", [1e-4, 5e-3, 0.2, 3.0])
def test_vxc_is_derivative_of_n_exc(n0):
    h = 1e-6 * n0
    ep, _ = xc.lda_xc(np.array([n0 + h]))
    em, _ = xc.lda_xc(np.array([n0 - h]))
    _, v = xc.lda_xc(np.array([n0]))
    fdv = ((n0 + h) * ep[0] - (n0 - h) * em[0]) / (2 * h)
    assert abs(fdv - v[0]) < 1e-8 * max(1, abs(v[0]))


def test_chi0_zero_temperature_limit():
    nbar = 0.01
    kf = (3 * math.pi ** 2 * nbar) ** (1 / 3)
    mu0 = 0.5 * kf * kf
    T = 1e-3 * mu0
    for q in (0.05, 0.4, 1.0, 2 * kf * 1.3, 3.0):
        a = chi0(q, mu0, T)
        b = chi0_zero_T(q, kf)
        assert abs(a - b) < 2e-5 * abs(b), (q, a, b)


@pytest.mark.parametrize("nbar,theta", [(0.0273, 0.5), (0.03, 1.0), (0.1, 0.1), (0.01, 2.0)])
def test_compressibility_sum_rule(nbar, theta):
    # -1/chi0(q -> 0) = d mu0/d n from the Fermi-Dirac integrals
    T = theta * 0.5 * (3 * math.pi ** 2 * nbar) ** (2 / 3)
    _, mu0, dmu = mean_density_params(nbar, T)
    q = 1e-4
    assert abs(-1 / chi0(q, mu0, T) - dmu) < 1e-6 * dmu


def _chi0_maldague(q, mu0, T):
    # chi0(q; T, mu0) = int dmu' chi0(q; T = 0, mu') / (4 T cosh^2((mu0 - mu')/(2T)))
    def f(m):
        kf = math.sqrt(2 * m)
        w = 1.0 / (4 * T * math.cosh((mu0 - m) / (2 * T)) ** 2)
        return chi0_zero_T(q, kf) * w
    hi = max(mu0, 0) + 60 * T
    brk = [x for x in (q * q / 8, mu0) if 0 < x < hi]
    return integrate.quad(f, 0.0, hi, points=brk or None, limit=400, epsabs=0, epsrel=1e-12)[0]


@pytest.mark.parametrize("q", [0.2, 0.9, 1.7, 3.5])
def test_chi0_matches_maldague_representation(q):
    nbar, theta = 0.0273, 0.5
    T = theta * 0.5 * (3 * math.pi ** 2 * nbar) ** (2 / 3)
    _, mu0, _ = mean_density_params(nbar, T)
    a = chi0(q, mu0, T)
    b = _chi0_maldague(q, mu0, T)
    assert abs(a - b) < 1e-9 * abs(b), (a, b)


def test_chi0_large_q():
    # -1/chi0 -> q^2 / (4 nbar) (free-particle limit)
    nbar, T = 0.0273, 0.2171
    _, mu0, _ = mean_density_params(nbar, T)
    q = 40.0
    assert abs(-1 / chi0(q, mu0, T) / (q * q / (4 * nbar)) - 1) < 1e-3


def test_kernel_wang_teter_limit():
    # theta -> 0: 2 a^2 nbar^(2a-2) K = (pi^2/kF) [1/F_L(eta) - 3 eta^2 - 1]
    nbar = 0.02
    kf = (3 * math.pi ** 2 * nbar) ** (1 / 3)
    T = 2e-4 * 0.5 * kf * kf
    _, mu0, dmu = mean_density_params(nbar, T)
    for q in (0.3, 1.0, 2.5):
        x = q / (2 * kf)
        FL = 0.5 + (1 - x * x) / (4 * x) * math.log(abs((1 + x) / (1 - x)))
        ref = math.pi ** 2 / kf * (1 / FL - 3 * x * x - 1) / (2 * ALPHA ** 2 * nbar ** (2 * ALPHA - 2))
        got = kernel_value(q, nbar, T, mu0, dmu)
        assert abs(got - ref) < 1e-4 * abs(ref), (q, got, ref)
    assert kernel_value(0.0, nbar, T, mu0, dmu) == 0.0


def test_kernel_large_q_limit_at_low_temperature():
    # For large eta = q/(2 kF), F_L = 1/(3 eta^2) + 1/(15 eta^4) + O(eta^-6), so
    # 1/F_L - 3 eta^2 - 1 -> -8/5: the kernel tends to -(8/5)(pi^2/kF) over
    # the prefactor 2 a^2 nbar^(2a-2), approached as 1/eta^2.
    nbar = 0.02
    kf = (3 * math.pi ** 2 * nbar) ** (1 / 3)
    T = 2e-4 * 0.5 * kf * kf
    _, mu0, dmu = mean_density_params(nbar, T)
    pref = 2 * ALPHA ** 2 * nbar ** (2 * ALPHA - 2)
    limit = -1.6 * math.pi ** 2 / kf / pref
    errs = []
    for eta in (4.0, 8.0):
        q = 2 * kf * eta
        FL = 0.5 + (1 - eta * eta) / (4 * eta) * math.log((eta + 1) / (eta - 1))
        exact = math.pi ** 2 / kf * (1 / FL - 3 * eta * eta - 1) / pref
        got = kernel_value(q, nbar, T, mu0, dmu)
        assert abs(got - exact) < 1e-6 * abs(exact), (eta, got, exact)
        errs.append(abs(got / limit - 1))
    # doubling eta divides the distance to the limit by about 4
    assert errs[1] < 2e-3 and 0.2 < errs[1] / errs[0] < 0.3

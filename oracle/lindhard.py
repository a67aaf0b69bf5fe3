"""Finite-temperature Lindhard response and the F_0^NL kernel of Eq. 2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

F_0^NL (Eq. 2) is a finite-temperature Wang-Teter functional whose kernel is
the second functional derivative of the free energy and depends only on the
mean valence density (Results, text after Eq. 2).  The paper prints neither the
exponents nor the kernel.  Reading used here (the Wang-Teter construction at
finite T):

  E_NL[n] = int int n^a(r) K(|r - r'|) n^a(r') dr dr'  (a = 1/2 by default,
            5/6 for the classic Wang-Teter choice; see functional.ALPHA_DEFAULT),
  2 a^2 nbar^(2a-2) K(q) = -1/chi0(q;T) - dmu0/dn - q^2 / (4 nbar),  K(0) = 0,

so that TF + vW + NL reproduce the ideal-gas static response at nbar.  chi0 is
the static Lindhard function of the ideal Fermi gas at temperature T:

  chi0(q;T) = -1/(pi^2 q) int_0^inf k f(k) ln|(2k + q)/(2k - q)| dk,
  f(k) = 1 / (1 + exp((k^2/2 - mu0)/T)),   mu0 = T eta(nbar).

The integral is done with SciPy's QUADPACK (quad), splitting at the
logarithmic singularity k = q/2 and using its algebraic-logarithmic weight
there.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

from .fermi_dirac import eta_from_density, fd_integral, PI2, SQRT2

ALPHA = 5.0 / 6.0   # Wang-Teter exponent (T -> 0 test reference); the functional's default is 1/2


def _occ(k, mu0, T):
    u = (0.5 * k * k - mu0) / T
    if u > 0:
        e = math.exp(-u)
        return e / (1.0 + e)
    return 1.0 / (1.0 + math.exp(u))


def _excess_integral(q: float, mu0: float, T: float) -> float:
    """I = int_0^inf k f(k) [ln|(2k+q)/(2k-q)| - 4k/q] dk.

    The leading large-q term 4k/q integrates to (4/q) pi^2 nbar exactly, so
    chi0 = -(4 nbar/q^2) (1 + eps) with eps = I q / (4 pi^2 nbar).  Working with
    I avoids subtracting two numbers of size q^2/(4 nbar) when the kernel is
    formed.  The integral is split around the Fermi edge sqrt(2 mu0) and at the
    logarithmic singularity q/2; on a piece that ends at q/2 the factor
    ln|k - q/2| is integrated with QUADPACK's algebraic-logarithmic weight.
    """
    kmax = math.sqrt(2.0 * max(mu0 + 45.0 * T, 45.0 * T))
    h = 0.5 * q
    opts = dict(epsabs=0.0, epsrel=1e-13, limit=400)
    brk = {0.0, kmax}
    # Fermi edge and points where (k^2/2 - mu0)/T = +-1, 3, 10, 30, so that the
    # drop of the occupation is never hidden between quadrature nodes
    for u in (-30.0, -10.0, -3.0, -1.0, 0.0, 1.0, 3.0, 10.0, 30.0):
        e = mu0 + u * T
        if e > 0 and math.sqrt(2.0 * e) < kmax:
            brk.add(math.sqrt(2.0 * e))
    if h < kmax:
        brk.add(h)
    pts = sorted(brk)
    g = lambda k: k * _occ(k, mu0, T)

    def excess(k):
        # ln|(1+x)/(1-x)| - 2x with x = 2k/q, written as 2(atanh x - x) below 1
        x = 2.0 * k / q
        if x < 1.0:
            return 2.0 * (math.atanh(x) - x)
        return math.log((x + 1.0) / (x - 1.0)) - 2.0 * x

    total = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        if b <= a:
            continue
        if a == h or b == h:
            # k f(k) [ln(2k + q) - ln 2 - 4k/q - ln|k - q/2|]
            reg = integrate.quad(lambda k: g(k) * (math.log(2.0 * k + q) - math.log(2.0) - 4.0 * k / q),
                                 a, b, **opts)[0]
            w = "alg-loga" if a == h else "alg-logb"
            sing = integrate.quad(g, a, b, weight=w, wvar=(0.0, 0.0), **opts)[0]
            total += reg - sing
        else:
            total += integrate.quad(lambda k: g(k) * excess(k), a, b, **opts)[0]
    return total


def chi0(q: float, mu0: float, T: float, nbar: float | None = None) -> float:
    """Static finite-T Lindhard function (negative), q > 0.  nbar is the
    ideal-gas density at (mu0, T); computed from the Fermi-Dirac integral when
    not given."""
    if nbar is None:
        nbar = float(SQRT2 / PI2 * T ** 1.5 * fd_integral(0.5, np.array([mu0 / T]))[0])
    eps = _excess_integral(q, mu0, T) * q / (4.0 * PI2 * nbar)
    return -4.0 * nbar / (q * q) * (1.0 + eps)


def response_excess(q: float, mu0: float, T: float, nbar: float) -> float:
    """-1/chi0(q) - q^2/(4 nbar) = -(q^2/(4 nbar)) eps/(1 + eps), formed
    without cancellation."""
    eps = _excess_integral(q, mu0, T) * q / (4.0 * PI2 * nbar)
    return -q * q / (4.0 * nbar) * eps / (1.0 + eps)


def chi0_zero_T(q: float, kf: float) -> float:
    """T = 0 Lindhard function -(kF/pi^2) F_L(q / 2kF), for tests."""
    x = q / (2.0 * kf)
    if abs(x - 1.0) < 1e-15:
        FL = 0.5
    else:
        FL = 0.5 + (1.0 - x * x) / (4.0 * x) * math.log(abs((1.0 + x) / (1.0 - x)))
    return -kf / PI2 * FL


def mean_density_params(nbar: float, T: float):
    """(eta0, mu0, dmu0/dn) of the ideal gas at the mean density."""
    eta0 = float(eta_from_density(np.array([nbar]), T)[0])
    im = float(fd_integral(-0.5, np.array([eta0]))[0])
    dmu = 2.0 * PI2 / (SQRT2 * math.sqrt(T) * im)
    return eta0, T * eta0, dmu


def kernel_value(q: float, nbar: float, T: float, mu0: float, dmu: float,
                 alpha: float = ALPHA) -> float:
    """K(q) from the response condition; K(0) = 0."""
    if q == 0.0:
        return 0.0
    return (response_excess(q, mu0, T, nbar) - dmu) / (2.0 * alpha * alpha * nbar ** (2 * alpha - 2))


def kernel_table(m2_values, L: float, nbar: float, T: float, alpha: float = ALPHA) -> np.ndarray:
    """K on integer shells: q = (2 pi / L) sqrt(m2) for each m2 in m2_values."""
    _, mu0, dmu = mean_density_params(nbar, T)
    out = np.empty(len(m2_values))
    for i, m2 in enumerate(m2_values):
        q = 2.0 * math.pi / L * math.sqrt(float(m2))
        out[i] = kernel_value(q, nbar, T, mu0, dmu, alpha)
    return out

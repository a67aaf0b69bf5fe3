"""Fermi-Dirac integrals and the finite-temperature Thomas-Fermi functional.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

F_s^TF[n;T] of Eq. 1 is named but not written out in the paper; the oracle uses
the textbook Feynman-Metropolis-Teller form for a spin-unpolarised ideal Fermi
gas (the TF functional "accurate in the high-density or high-temperature
limit", Results, after Eq. 1):

    I_nu(eta)  = int_0^inf x^nu / (1 + exp(x - eta)) dx
    n          = sqrt(2)/pi^2 * T^(3/2) * I_{1/2}(eta)
    f_TF(n;T)  = n T eta - 2 sqrt(2)/(3 pi^2) * T^(5/2) * I_{3/2}(eta)
    v_TF       = d f_TF / d n = T eta

The integrals are done by composite Gauss-Legendre quadrature in t = sqrt(x)
and eta(n) by bracketed Newton iteration, both in oracle/fdint.c (plain C,
OpenMP over grid points).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from ._native import lib

SQRT2 = math.sqrt(2.0)
PI2 = math.pi ** 2
_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def fd_integrals(eta):
    """(I_{-1/2}, I_{1/2}, I_{3/2}) at eta, each with eta's shape."""
    e = np.ascontiguousarray(np.asarray(eta, dtype=float))
    flat = e.ravel()
    im = np.empty_like(flat)
    ih = np.empty_like(flat)
    i3 = np.empty_like(flat)
    lib().oracle_fd_integrals(_ptr(flat), flat.size, _ptr(im), _ptr(ih), _ptr(i3))
    return im.reshape(e.shape), ih.reshape(e.shape), i3.reshape(e.shape)


def fd_integral(nu: float, eta):
    """I_nu(eta) for nu in {-1/2, 1/2, 3/2}."""
    k = {-0.5: 0, 0.5: 1, 1.5: 2}[float(nu)]
    return fd_integrals(eta)[k]


def inverse_fd_half(y, eta0=None, tol: float = 1e-14):
    """eta with I_{1/2}(eta) = y (y > 0).  eta0 is only a starting guess."""
    yy = np.ascontiguousarray(np.asarray(y, dtype=float))
    flat = yy.ravel()
    out = np.empty_like(flat)
    g = None
    if eta0 is not None:
        g = np.ascontiguousarray(np.asarray(eta0, dtype=float).ravel())
        if g.size != flat.size:
            g = None
    bad = lib().oracle_fd_inverse_half(_ptr(flat), flat.size,
                                       _ptr(g) if g is not None else None,
                                       _ptr(out), tol)
    if bad:
        raise RuntimeError(f"inverse_fd_half: {bad} points did not converge")
    return out.reshape(yy.shape)


def reduced_density(n, T: float):
    """y = pi^2 n / (sqrt2 T^(3/2)) = I_{1/2}(eta)."""
    return PI2 * np.asarray(n, dtype=float) / (SQRT2 * T ** 1.5)


def density_from_eta(eta, T: float):
    """n(eta) = sqrt(2)/pi^2 T^(3/2) I_{1/2}(eta)."""
    return SQRT2 / PI2 * T ** 1.5 * fd_integral(0.5, eta)


def eta_from_density(n, T: float, eta0=None):
    """Reduced chemical potential eta(n, T)."""
    return inverse_fd_half(reduced_density(n, T), eta0=eta0)


def tf_free_energy_density(n, T: float, eta0=None):
    """(f_TF, v_TF, eta) pointwise for the finite-T Thomas-Fermi functional."""
    n = np.asarray(n, dtype=float)
    eta = eta_from_density(n, T, eta0=eta0)
    i32 = fd_integral(1.5, eta)
    f = n * T * eta - 2.0 * SQRT2 / (3.0 * PI2) * T ** 2.5 * i32
    return f, T * eta, eta


def dmu_dn(n: float, T: float) -> float:
    """d mu/d n of the ideal gas: 2 pi^2 / (sqrt2 T^(1/2) I_{-1/2}(eta))."""
    eta = eta_from_density(np.array([n]), T)
    im = float(fd_integral(-0.5, eta)[0])
    return 2.0 * PI2 / (SQRT2 * math.sqrt(T) * im)

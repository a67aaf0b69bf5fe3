"""Grid, reciprocal vectors, structure factor, local pseudopotential, Ewald.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (Hartree atomic units, cubic cell of side L, Omega = L^3, n^3 grid
points r = (L/n) * (i, j, k)):

* G = (2 pi / L) m with integer m in FFT order (np.fft.fftfreq); on even grids
  the Nyquist index carries m = -n/2.
* f~(G) = (1/N) sum_r f(r) exp(-i G.r)  (numpy fftn divided by N = n^3), so
  f(r) = sum_G f~(G) exp(i G.r) and int f* g = Omega sum_G f~* g~.
* Ion structure factor S(G) = sum_I exp(-i G.R_I): the reciprocal-space ion
  density n_i(q) of the paper's S_ab definition (Methods, static structure
  factors).
* Local pseudopotential: the paper uses Heine-Abarenkov (H) and a local
  norm-conserving table (Be) whose parameters it does not print (Methods).
  Reading: a Gaussian-smoothed Coulomb ion, v(r) = -Z erf(r/rc)/r, whose
  transform is v~(G) = -4 pi Z exp(-G^2 rc^2/4) / G^2; at G = 0 the
  non-Coulomb remainder of (v + Z/r) integrates to pi Z rc^2.
  V_loc(G) = (1/Omega) sum_I v~_I(G) exp(-i G.R_I).
* Ion-ion energy: point charges Z_I in a neutralising background (Ewald), the
  same G = 0 convention under which Hartree drops its G = 0 term.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import erfc


def integer_m(n: int) -> np.ndarray:
    """Integer wave numbers in FFT order."""
    return np.rint(np.fft.fftfreq(n) * n).astype(np.int64)


def m2_grid(n: int) -> np.ndarray:
    """|m|^2 on the full n^3 FFT grid (int64)."""
    m = integer_m(n)
    return m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2


def g2_grid(n: int, L: float) -> np.ndarray:
    return (2.0 * math.pi / L) ** 2 * m2_grid(n).astype(float)


def structure_factor(pos: np.ndarray, n: int, L: float, weights=None) -> np.ndarray:
    """S(G) = sum_I w_I exp(-i G.R_I) on the full FFT grid (complex128)."""
    m = integer_m(n)
    pos = np.asarray(pos, dtype=float)
    w = np.ones(len(pos)) if weights is None else np.asarray(weights, dtype=float)
    S = np.zeros((n, n, n), dtype=complex)
    for I in range(len(pos)):
        ph = [np.exp(-2j * math.pi * m * pos[I, d] / L) for d in range(3)]
        S += w[I] * ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
    return S


def vloc_g(Z: np.ndarray, pos: np.ndarray, n: int, L: float, rc: float) -> np.ndarray:
    """V_loc(G) of the Gaussian-smoothed Coulomb ions (complex, full grid)."""
    G2 = g2_grid(n, L)
    Z = np.asarray(Z, dtype=float)
    Omega = L ** 3
    out = np.zeros((n, n, n), dtype=complex)
    for z in np.unique(Z):
        sel = Z == z
        S = structure_factor(pos[sel], n, L)
        with np.errstate(divide="ignore", invalid="ignore"):
            vt = np.where(G2 > 0, -4.0 * math.pi * z * np.exp(-G2 * rc * rc / 4.0) / G2, 0.0)
        vt[0, 0, 0] = math.pi * z * rc * rc
        out += vt * S / Omega
    return out


def ewald_energy(Z: np.ndarray, pos: np.ndarray, L: float, eta: float | None = None,
                 tol: float = 1e-16) -> float:
    """Ewald energy of point charges Z_I in a uniform neutralising background.

    E = 1/2 sum_{I,J} sum_R' Z_I Z_J erfc(eta |R_IJ + R|)/|R_IJ + R|
      + (2 pi / Omega) sum_{G != 0} exp(-G^2/(4 eta^2)) / G^2 |sum_I Z_I e^{iG.R_I}|^2
      - eta/sqrt(pi) sum_I Z_I^2 - pi (sum_I Z_I)^2 / (2 Omega eta^2)
    The result does not depend on the splitting parameter eta.
    """
    Z = np.asarray(Z, dtype=float)
    pos = np.asarray(pos, dtype=float)
    Omega = L ** 3
    if eta is None:
        eta = math.sqrt(math.pi) / L * 2.0
    # real-space cutoff: erfc(eta r) < tol
    rcut = 1.0
    while erfc(eta * rcut) / rcut > tol:
        rcut *= 1.1
    nimg = int(math.ceil(rcut / L)) + 1
    e_real = 0.0
    shifts = np.array(list(itertools.product(range(-nimg, nimg + 1), repeat=3)), float) * L
    for I in range(len(Z)):
        d = pos[I][None, :] - pos                      # [J, 3]
        r = np.linalg.norm(d[:, None, :] + shifts[None, :, :], axis=2)   # [J, S]
        mask = (r > 1e-12) & (r < rcut)
        e_real += 0.5 * Z[I] * np.sum((Z[:, None] * erfc(eta * r) / np.where(mask, r, 1.0))[mask])
    # reciprocal space: exp(-G^2/(4 eta^2)) < tol
    gcut = 2.0 * eta * math.sqrt(-math.log(tol))
    mmax = int(math.ceil(gcut * L / (2.0 * math.pi)))
    rng = np.arange(-mmax, mmax + 1)
    mx, my, mz = np.meshgrid(rng, rng, rng, indexing="ij")
    G = 2.0 * math.pi / L * np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1).astype(float)
    G2 = np.sum(G * G, axis=1)
    keep = (G2 > 0) & (G2 <= gcut * gcut)
    G = G[keep]
    G2 = G2[keep]
    S = np.zeros(len(G), dtype=complex)
    for I in range(len(Z)):
        S += Z[I] * np.exp(1j * G @ pos[I])
    e_recip = 2.0 * math.pi / Omega * np.sum(np.exp(-G2 / (4.0 * eta * eta)) / G2 * np.abs(S) ** 2)
    e_self = -eta / math.sqrt(math.pi) * np.sum(Z * Z)
    e_bg = -math.pi * np.sum(Z) ** 2 / (2.0 * Omega * eta * eta)
    return float(e_real + e_recip + e_self + e_bg)

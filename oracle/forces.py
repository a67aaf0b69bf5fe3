"""Hellmann-Feynman forces on the ions at a given density.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

At fixed electron density n the free energy depends on the ion positions only
through the electron-ion term E_loc and the ion-ion Ewald energy (the other
terms are functionals of n alone), so the force on ion I is

    F_I = -dE_loc/dR_I - dE_ion/dR_I.

With V_loc(G) = (1/Omega) sum_J v~_J(G) exp(-i G.R_J) and
E_loc = Omega sum_G Re[n~*(G) V_loc(G)] (full G sum):

    F_I(loc) = -sum_G G v~_I(G) Im[n~*(G) exp(-i G.R_I)].

For the Ewald energy of oracle.cell.ewald_energy (splitting eta):

    F_I(real)  = sum_J sum_R' Z_I Z_J [erfc(eta r)/r^2 + 2 eta/sqrt(pi) exp(-eta^2 r^2)/r] d/r,
                 d = R_I - R_J + R, r = |d|,
    F_I(recip) = (4 pi / Omega) Z_I sum_{G != 0} exp(-G^2/(4 eta^2))/G^2 G Im[A(G) exp(i G.R_I)],
                 A(G) = sum_J Z_J exp(-i G.R_J).

Within the paper these forces drive the molecular dynamics that produces its
structure factors (Methods); they are the derivative of the energy the hot
path minimises, and the tests pin them to finite differences of that energy.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import erfc

from .cell import integer_m, g2_grid
from .functional import fft3


def local_forces(Z, pos, rho, L, rc) -> np.ndarray:
    """-dE_loc/dR_I at fixed density rho (n^3 real grid); returns [N_ion, 3]."""
    n = rho.shape[0]
    nt = fft3(rho)
    m = integer_m(n)
    tp = 2.0 * math.pi / L
    G2 = g2_grid(n, L)
    Gx = tp * m[:, None, None] * np.ones((1, n, n))
    Gy = tp * m[None, :, None] * np.ones((n, 1, n))
    Gz = tp * m[None, None, :] * np.ones((n, n, 1))
    out = np.zeros((len(Z), 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        base = np.where(G2 > 0, -4.0 * math.pi * np.exp(-G2 * rc * rc / 4.0) / G2, 0.0)
    for I in range(len(Z)):
        ph = [np.exp(-1j * tp * m * pos[I, d]) for d in range(3)]
        e = ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
        im = np.imag(np.conj(nt) * e) * (Z[I] * base)
        out[I] = [-np.sum(Gx * im), -np.sum(Gy * im), -np.sum(Gz * im)]
    return out


def ewald_forces(Z, pos, L, eta=None, tol=1e-16) -> np.ndarray:
    """-dE_ion/dR_I of oracle.cell.ewald_energy; returns [N_ion, 3]."""
    Z = np.asarray(Z, dtype=float)
    pos = np.asarray(pos, dtype=float)
    Omega = L ** 3
    if eta is None:
        eta = math.sqrt(math.pi) / L * 2.0
    rcut = 1.0
    while erfc(eta * rcut) / rcut > tol:
        rcut *= 1.1
    nimg = int(math.ceil(rcut / L)) + 1
    shifts = np.array(list(itertools.product(range(-nimg, nimg + 1), repeat=3)), float) * L
    out = np.zeros((len(Z), 3))
    for I in range(len(Z)):
        d = pos[I][None, None, :] - pos[:, None, :] + shifts[None, :, :]     # [J, S, 3]
        r = np.linalg.norm(d, axis=2)
        mask = (r > 1e-12) & (r < rcut)
        rr = np.where(mask, r, 1.0)
        f = (erfc(eta * rr) / rr ** 2 + 2.0 * eta / math.sqrt(math.pi) * np.exp(-(eta * rr) ** 2) / rr) / rr
        f = np.where(mask, f, 0.0) * Z[I] * Z[:, None]
        out[I] += np.sum(f[:, :, None] * d, axis=(0, 1))
    gcut = 2.0 * eta * math.sqrt(-math.log(tol))
    mmax = int(math.ceil(gcut * L / (2.0 * math.pi)))
    rng = np.arange(-mmax, mmax + 1)
    mx, my, mz = np.meshgrid(rng, rng, rng, indexing="ij")
    G = 2.0 * math.pi / L * np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1).astype(float)
    G2 = np.sum(G * G, axis=1)
    keep = (G2 > 0) & (G2 <= gcut * gcut)
    G, G2 = G[keep], G2[keep]
    A = np.zeros(len(G), dtype=complex)
    for J in range(len(Z)):
        A += Z[J] * np.exp(-1j * G @ pos[J])
    w = np.exp(-G2 / (4.0 * eta * eta)) / G2
    for I in range(len(Z)):
        im = np.imag(A * np.exp(1j * G @ pos[I]))
        out[I] += 4.0 * math.pi / Omega * Z[I] * np.sum((w * im)[:, None] * G, axis=0)
    return out


def forces(cell, rho) -> np.ndarray:
    """Hellmann-Feynman forces [N_ion, 3] at density rho for a workloads.Cell."""
    Z = np.asarray(cell.Z, dtype=float)
    pos = np.asarray(cell.pos, dtype=float)
    return local_forces(Z, pos, rho, cell.L, cell.rc) + ewald_forces(Z, pos, cell.L)

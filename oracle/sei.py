"""Electron-ion and ion-ion static structure factors on |q| shells.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Methods, static structure factors: S_ab(q) = (1/sqrt(N_a N_b)) <n_a(q) n_b*(q)>,
averaged over wave vectors of equal magnitude (and over MD steps; one snapshot
here).  With a = e (electrons), b = i (ions):

  n_e(G) = int n(r) exp(-i G.r) dr = Omega n~(G),  n_i(G) = S(G) = sum_I exp(-i G.R_I)
  S_ei(q_k) = (1/sqrt(N_e N_i)) * mean over {G : |m|^2 = m2_k} of Re[n_e(G) S*(G)]

Shells are the distinct nonzero integer |m|^2 present on the full FFT grid
(exact equal-|q| shells), in ascending order.
"""
from __future__ import annotations

import math

import numpy as np

from .cell import m2_grid, structure_factor
from .functional import fft3


def sei_shells(rho: np.ndarray, pos: np.ndarray, L: float, n_electrons: float, n_shells: int = 200):
    n = rho.shape[0]
    Omega = L ** 3
    ne = Omega * fft3(rho)
    ni = structure_factor(pos, n, L)
    prod = (ne * np.conj(ni)).real
    m2 = m2_grid(n)
    values = np.unique(m2[m2 > 0])[:n_shells]
    q = 2.0 * math.pi / L * np.sqrt(values.astype(float))
    s = np.array([prod[m2 == v].mean() for v in values]) / math.sqrt(n_electrons * len(pos))
    return q, s


def sii_shells(pos: np.ndarray, L: float, n: int, n_shells: int = 200):
    """Ion-ion static structure factor on the same shells:
    S_ii(q_k) = (1/N_i) * mean over {G : |m|^2 = m2_k} of |S(G)|^2 (Methods,
    S_ab with a = b = i, one snapshot)."""
    ni = structure_factor(pos, n, L)
    m2 = m2_grid(n)
    values = np.unique(m2[m2 > 0])[:n_shells]
    q = 2.0 * math.pi / L * np.sqrt(values.astype(float))
    p2 = np.abs(ni) ** 2
    s = np.array([p2[m2 == v].mean() for v in values]) / len(pos)
    return q, s


def sei_shells_direct(rho: np.ndarray, pos: np.ndarray, L: float, n_electrons: float, n_shells: int = 200):
    """sei_shells for large cells: the same definition, with S(G) summed
    directly over the ions only for the wave vectors of the requested shells
    (the full-grid structure factor of ~1000 ions on 256^3 is out of reach on
    a CPU).  n_e(G) still comes from the full transform of rho."""
    n = rho.shape[0]
    Omega = L ** 3
    ne = Omega * fft3(rho)
    m2 = m2_grid(n)
    values = np.unique(m2[m2 > 0])[:n_shells]
    q = 2.0 * math.pi / L * np.sqrt(values.astype(float))
    m = np.rint(np.fft.fftfreq(n) * n).astype(np.int64)
    s = np.empty(len(values))
    pos = np.asarray(pos, dtype=float)
    # the grid vectors of all requested shells in one scan, grouped by m^2
    flat = m2.ravel()
    sel = np.nonzero((flat > 0) & (flat <= values[-1]))[0]
    sel = sel[np.argsort(flat[sel], kind="stable")]
    bounds = np.searchsorted(flat[sel], np.concatenate([values, [values[-1] + 1]]))
    for i in range(len(values)):
        ix, iy, iz = np.unravel_index(sel[bounds[i]:bounds[i + 1]], m2.shape)
        G = 2.0 * math.pi / L * np.stack([m[ix], m[iy], m[iz]], axis=1).astype(float)
        S = np.exp(-1j * (G @ pos.T)).sum(axis=1)
        s[i] = float(np.mean((ne[ix, iy, iz] * np.conj(S)).real))
    return q, s / math.sqrt(n_electrons * len(pos))

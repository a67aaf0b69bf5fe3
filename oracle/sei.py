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


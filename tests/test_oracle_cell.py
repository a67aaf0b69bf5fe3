"""Pins of the structure factor, local pseudopotential and Ewald energy."""
import math

import numpy as np
from scipy.special import erf

from oracle.cell import ewald_energy, structure_factor, vloc_g, integer_m, g2_grid
from oracle.functional import ifft3
from workloads import fcc_cell, random_cell


def test_ewald_independent_of_splitting():
    c = random_cell(11, 6, 1.0, 1.5, 1.0, 16)
    e = [ewald_energy(c.Z, c.pos, c.L, eta) for eta in (0.4, 0.7, 1.1, 1.6)]
    assert max(e) - min(e) < 1e-11 * abs(e[0])


def test_ewald_fcc_madelung():
    # fcc lattice of point charges in a neutralising background (one-component
    # plasma): E/N = -0.895873615195 Z^2 / a_WS (the fcc Madelung constant)
    for a, Z in ((7.6, 3.0), (3.3, 1.0)):
        c = fcc_cell(a=a, Z=Z)
        aws = (3 * a ** 3 / (4 * math.pi * 4)) ** (1 / 3)
        e = ewald_energy(c.Z, c.pos, c.L) / 4
        assert abs(e / (Z * Z / aws) + 0.895873615195) < 1e-10


def test_structure_factor_direct_sum():
    c = random_cell(5, 3, 1.0, 1.0, 1.0, 8)
    S = structure_factor(c.pos, 8, c.L)
    m = integer_m(8)
    for (i, j, k) in ((1, 2, 3), (7, 0, 4), (5, 5, 5)):
        G = 2 * math.pi / c.L * np.array([m[i], m[j], m[k]])
        ref = sum(np.exp(-1j * G @ p) for p in c.pos)
        assert abs(S[i, j, k] - ref) < 1e-12


def test_vloc_single_ion_real_space():
    # one ion at the cell centre: v(r) = sum over images of -Z erf(r/rc)/r, up to
    # the constant fixed by the G = 0 convention; compare differences of v
    L, n, rc, Z = 12.0, 48, 1.0, 2.0
    pos = np.array([[L / 2, L / 2, L / 2]])
    v = ifft3(vloc_g(np.array([Z]), pos, n, L, rc))
    h = L / n
    pts = [(24, 24, 24), (24, 24, 30), (24, 30, 30), (30, 30, 30)]

    def direct(p):
        r0 = np.array(p) * h
        tot = 0.0
        # Ewald-free check: smooth short-range part plus long-range Coulomb sum
        # converges slowly, so use the difference of two points which only
        # needs near images
        for a in range(-2, 3):
            for b in range(-2, 3):
                for cc in range(-2, 3):
                    d = np.linalg.norm(r0 - pos[0] - L * np.array([a, b, cc]))
                    tot += -Z * erf(d / rc) / d if d > 1e-12 else -Z * 2 / (math.sqrt(math.pi) * rc)
        return tot
    ref = [direct(p) for p in pts]
    got = [v[p] for p in pts]
    # differences between nearby points are dominated by the central ion
    for k in range(1, len(pts)):
        assert abs((got[k] - got[0]) - (ref[k] - ref[0])) < 2e-2


def test_vloc_uniform_energy():
    c = random_cell(3, 5, 3.0, 1.5, 1.0, 16)
    V = vloc_g(c.Z, c.pos, 16, c.L, c.rc)
    nbar = c.n_electrons / c.volume
    e_loc = c.volume * (nbar * V[0, 0, 0]).real
    assert abs(e_loc - nbar * np.sum(math.pi * c.Z * c.rc ** 2)) < 1e-12

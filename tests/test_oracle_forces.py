"""Pins of the oracle's Hellmann-Feynman forces: at fixed density the force is
minus the derivative of the free energy with respect to the ion positions, so
central finite differences of the oracle energy (rebuilt at displaced ions)
fix every component; the Ewald part also obeys sum_I F_I = 0."""
import math

import numpy as np
import pytest

from oracle.functional import Functional
from oracle.cell import ewald_energy
from oracle.forces import forces, ewald_forces, local_forces
from workloads import random_cell, fcc_cell
from workloads.cells import Cell


def _displaced(cell, I, d, h):
    pos = np.array(cell.pos, dtype=float).copy()
    pos[I, d] += h
    return Cell(L=cell.L, n=cell.n, Z=cell.Z, pos=pos, theta=cell.theta, rc=cell.rc, label=cell.label)


def _density(cell, seed=3):
    rng = np.random.default_rng(seed)
    n = cell.n
    x = np.arange(n) / n
    sm = sum(rng.uniform(0.2, 1.0) * np.cos(2 * math.pi * (k[0] * x[:, None, None] + k[1] * x[None, :, None]
                                                               + k[2] * x[None, None, :]) + rng.uniform(0, 6.28))
             for k in rng.integers(-3, 4, size=(5, 3)))
    rho = np.exp(0.3 * sm / 3.0)
    return rho * cell.n_electrons / (rho.sum() * cell.volume / rho.size)


def test_ewald_forces_match_energy_differences_and_sum_to_zero():
    c = random_cell(31, 6, 3.0, 1.8, 1.0, 16)
    Z = np.asarray(c.Z, float)
    F = ewald_forces(Z, c.pos, c.L)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-10 * max(1.0, np.abs(F).max())
    h = 1e-5
    for I, d in ((0, 0), (2, 1), (5, 2)):
        p1 = np.array(c.pos, float); p1[I, d] += h
        p0 = np.array(c.pos, float); p0[I, d] -= h
        fd = -(ewald_energy(Z, p1, c.L) - ewald_energy(Z, p0, c.L)) / (2 * h)
        assert abs(fd - F[I, d]) < 1e-6 * max(1.0, abs(F[I, d]))


@pytest.mark.parametrize("mk", [lambda: random_cell(32, 5, 1.0, 1.7, 0.8, 20), lambda: fcc_cell(n=16)])
def test_total_forces_match_energy_differences_at_fixed_density(mk):
    c = mk()
    rho = _density(c)
    F = forces(c, rho)
    h = 1e-5
    for I, d in ((0, 0), (1, 2), (len(c.Z) - 1, 1)):
        e1 = Functional(_displaced(c, I, d, h)).evaluate(rho)[0]["total"]
        e0 = Functional(_displaced(c, I, d, -h)).evaluate(rho)[0]["total"]
        fd = -(e1 - e0) / (2 * h)
        assert abs(fd - F[I, d]) < 2e-6 * max(1.0, abs(F[I, d])), (I, d, fd, F[I, d])


def test_local_force_of_a_uniform_density_vanishes():
    c = random_cell(33, 4, 1.0, 2.0, 1.0, 16)
    rho = np.full((16,) * 3, c.n_electrons / c.volume)
    F = local_forces(np.asarray(c.Z, float), c.pos, rho, c.L, c.rc)
    assert np.max(np.abs(F)) < 1e-12

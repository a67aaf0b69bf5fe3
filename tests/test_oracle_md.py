"""Pins of the oracle's ion dynamics (oracle/md.py): the velocity-Verlet
orbit of a harmonic oscillator in closed form, time reversibility and the
O(dt^2) conservation of the Nose-Hoover extended energy on an anharmonic
many-body system, and, for OFDFT ions, the Hellmann-Feynman theorem (the force
at the electronic minimum is minus the total derivative of the minimised free
energy) and energy conservation of a short NVE run."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import md
from oracle.functional import Functional
from oracle.minimize import lbfgs
from oracle.forces import forces
from workloads import random_cell


def test_velocity_verlet_harmonic_orbit_closed_form():
    # x_n = x0 cos(n w~ dt) with cos(w~ dt) = 1 - (w dt)^2 / 2 exactly
    m, k, dt = 2.0, 3.0, 0.3
    w = math.sqrt(k / m)
    x0 = np.array([[0.7, -0.2, 0.4]])
    st = md.MDState(pos=x0.copy(), vel=np.zeros((1, 3)))
    frames = md.run(st, [m], lambda p, _: (0.5 * k * float(np.sum(p * p)), -k * p, None), 50, dt)
    wt = math.acos(1.0 - 0.5 * (w * dt) ** 2) / dt
    for i, f in enumerate(frames, start=1):
        assert np.allclose(f.pos, x0 * math.cos(i * wt * dt), atol=1e-12, rtol=0)


def _anharmonic():
    # 5 particles: quartic confinement plus soft pair repulsion (chaotic)
    rng = np.random.default_rng(4)
    pos = rng.uniform(-1, 1, size=(5, 3))
    vel = rng.normal(0, 0.3, size=(5, 3))
    vel -= vel.mean(axis=0)
    mass = np.array([1.0, 2.0, 1.5, 1.0, 3.0])

    def fn(p, _):
        e = 0.25 * float(np.sum(p ** 4))
        f = -p ** 3
        for i in range(len(p)):
            for j in range(i + 1, len(p)):
                d = p[i] - p[j]
                r2 = float(d @ d)
                e += math.exp(-r2)
                fij = 2.0 * math.exp(-r2) * d
                f[i] += fij
                f[j] -= fij
        return e, f, None
    return pos, vel, mass, fn


def test_nose_hoover_is_time_reversible():
    pos, vel, mass, fn = _anharmonic()
    st = md.MDState(pos=pos.copy(), vel=vel.copy(), xi=0.05)
    md.run(st, mass, fn, 300, 0.02, T=0.2, tau=1.0)
    st.vel = -st.vel
    st.xi = -st.xi
    md.run(st, mass, fn, 300, 0.02, T=0.2, tau=1.0)
    assert np.abs(st.pos - pos).max() < 1e-9
    assert np.abs(st.vel + vel).max() < 1e-9
    assert abs(st.xi + 0.05) < 1e-9 and abs(st.s) < 1e-9


@pytest.mark.parametrize("thermostat", [False, True])
def test_extended_energy_error_is_second_order(thermostat):
    pos, vel, mass, fn = _anharmonic()
    kw = dict(T=0.2, tau=1.0) if thermostat else {}
    dev = []
    for dt in (0.02, 0.01):
        st = md.MDState(pos=pos.copy(), vel=vel.copy())
        fr = md.run(st, mass, fn, int(round(20 / dt)), dt, **kw)
        H = np.array([f.conserved for f in fr])
        dev.append(np.abs(H - H[0]).max())
    assert dev[0] < 1e-3
    assert 3.0 < dev[0] / dev[1] < 5.0


def test_thermostat_exchanges_energy():
    # g T above 2K: the friction goes negative and heats the ions
    pos, vel, mass, fn = _anharmonic()
    st = md.MDState(pos=pos.copy(), vel=vel.copy())
    K0 = md.kinetic(vel, mass)
    T = 4.0 * 2.0 * K0 / (3 * len(mass) - 3)
    fr = md.run(st, mass, fn, 200, 0.01, T=T, tau=0.5)
    assert fr[0].xi < 0
    assert max(f.kinetic for f in fr) > 1.5 * K0


@pytest.fixture(scope="module")
def tiny_cell():
    return random_cell(51, 3, 1.0, 1.6, 1.0, 12)


def test_hellmann_feynman_force_is_total_derivative(tiny_cell):
    cell = tiny_cell
    K = Functional(cell).K

    def fmin(pos):
        c = replace(cell, pos=pos)
        r = lbfgs(Functional(c, kernel=K), tol_F=1e-13, tol_R=1e-10, max_iter=4000)
        assert r.converged
        return c, r

    c0, r0 = fmin(np.asarray(cell.pos, float))
    F = forces(c0, r0.rho)
    h = 1e-3
    for I, d in ((0, 0), (1, 2), (2, 1)):
        e = []
        for s in (1, -1):
            p = np.asarray(cell.pos, float).copy()
            p[I, d] += s * h
            e.append(fmin(p)[1].energies["total"])
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - F[I, d]) < 1e-5 * max(1.0, abs(F).max()), (I, d, fd, F[I, d])


def test_ofdft_nve_conserves_energy(tiny_cell):
    cell = tiny_cell
    mass = np.full(cell.n_ion, 1836.15267)
    rng = np.random.default_rng(3)
    vel = rng.normal(0, math.sqrt(0.01 / 1836.15267), size=(cell.n_ion, 3))
    vel -= vel.mean(axis=0)
    st = md.MDState(pos=np.asarray(cell.pos, float).copy(), vel=vel)
    fr = md.run(st, mass, md.ofdft_force_fn(cell), 8, 10.0, L=cell.L)
    H = np.array([f.conserved for f in fr])
    K = np.array([f.kinetic for f in fr])
    assert np.abs(H - H[0]).max() < 2e-2 * (K.max() - K.min() + 1e-12) + 1e-7


def test_thermostat_rests_at_equipartition_with_g_3n_minus_3():
    # free ions with zero total momentum and 2K = (3N - 3) T: the friction
    # has nothing to correct and stays zero (the reading of g)
    rng = np.random.default_rng(8)
    vel = rng.normal(size=(6, 3))
    vel -= vel.mean(axis=0)
    mass = np.ones(6)
    T = 2.0 * md.kinetic(vel, mass) / (3 * 6 - 3)
    st = md.MDState(pos=np.zeros((6, 3)), vel=vel.copy())
    fr = md.run(st, mass, lambda p, _: (0.0, np.zeros_like(p), None), 20, 0.1, T=T, tau=1.0)
    assert max(abs(f.xi) for f in fr) < 1e-13
    assert np.allclose(st.vel, vel, rtol=0, atol=1e-13)

"""Born-Oppenheimer molecular dynamics of the ions with a Nose-Hoover thermostat.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's structure factors and pressures come from OFDFT molecular dynamics
in the NVT ensemble with a Nose-Hoover thermostat (Methods, "Molecular
dynamics": time steps of 0.1, 0.02 and 0.003 fs, thousands of equilibration
steps, then sampled steps).  It prints neither the integrator nor the
thermostat mass.  Reading used here: one Nose-Hoover variable xi (friction)
with mass Q, degrees of freedom g = 3 N_i - 3 (total momentum zero), and the
symmetric Trotter splitting

    NH(dt/2)  v += (dt/2) F/m  x += dt v  [new F]  v += (dt/2) F/m  NH(dt/2),

    NH(h):  xi += (h/2) (2K - g T)/Q;  v *= exp(-xi h);  s += xi h;
            xi += (h/2) (2K - g T)/Q          (K the kinetic energy at that moment)

which is time reversible and conserves H = E_pot + K + Q xi^2/2 + g T s to
O(dt^2).  Q = g T tau^2 for a thermostat period tau.  Without a thermostat
(T is None) the step is plain velocity Verlet (NVE).  Every step the electrons
are minimised at the new ion positions (E_pot = F_min, force = Hellmann-Feynman
force), starting from the previous step's density.  Positions are kept inside
[0, L) (the physics is periodic).  Atomic units: time in hbar/E_h, masses in
electron masses.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MDState:
    pos: np.ndarray          # [N, 3] bohr
    vel: np.ndarray          # [N, 3] bohr / (hbar/E_h)
    xi: float = 0.0          # thermostat friction
    s: float = 0.0           # thermostat position (integral of xi), for H
    forces: np.ndarray | None = None
    e_pot: float | None = None
    payload: object = None   # e.g. the converged density (warm start)


@dataclass
class MDFrame:
    e_pot: float
    kinetic: float
    xi: float
    s: float
    conserved: float
    pos: np.ndarray
    vel: np.ndarray


def kinetic(vel, mass) -> float:
    return 0.5 * float(np.sum(mass[:, None] * vel * vel))


def _nh_half(vel, mass, xi, s, h, T, Q, g):
    K = kinetic(vel, mass)
    xi += 0.5 * h * (2.0 * K - g * T) / Q
    vel = vel * math.exp(-xi * h)
    s += xi * h
    K = kinetic(vel, mass)
    xi += 0.5 * h * (2.0 * K - g * T) / Q
    return vel, xi, s


def run(state: MDState, mass, force_fn, n_steps: int, dt: float, L: float | None = None,
        T: float | None = None, tau: float | None = None, g: int | None = None) -> list[MDFrame]:
    """Advance `state` by n_steps.  force_fn(pos, payload) -> (e_pot, forces, payload).
    Returns one frame per step (after the step)."""
    mass = np.asarray(mass, dtype=float)
    n = len(mass)
    if g is None:
        g = 3 * n - 3
    thermo = T is not None
    Q = g * T * tau * tau if thermo else 0.0
    if state.forces is None:
        state.e_pot, state.forces, state.payload = force_fn(state.pos, state.payload)
    pos, vel, xi, s = state.pos.copy(), state.vel.copy(), state.xi, state.s
    F = state.forces
    frames = []
    for _ in range(n_steps):
        if thermo:
            vel, xi, s = _nh_half(vel, mass, xi, s, 0.5 * dt, T, Q, g)
        vel = vel + 0.5 * dt * F / mass[:, None]
        pos = pos + dt * vel
        if L is not None:
            pos = pos - L * np.floor(pos / L)
        e_pot, F, state.payload = force_fn(pos, state.payload)
        vel = vel + 0.5 * dt * F / mass[:, None]
        if thermo:
            vel, xi, s = _nh_half(vel, mass, xi, s, 0.5 * dt, T, Q, g)
        K = kinetic(vel, mass)
        H = e_pot + K + (0.5 * Q * xi * xi + g * T * s if thermo else 0.0)
        frames.append(MDFrame(e_pot, K, xi, s, H, pos.copy(), vel.copy()))
    state.pos, state.vel, state.xi, state.s, state.forces, state.e_pot = pos, vel, xi, s, F, e_pot
    return frames


def ofdft_force_fn(cell, minimize_kwargs=None):
    """force_fn for run(): minimise the oracle functional at the given ion
    positions (warm start from the previous density) and return
    (F_min, Hellmann-Feynman forces, density)."""
    from dataclasses import replace
    from .functional import Functional
    from .minimize import lbfgs
    from .forces import forces
    kw = dict(tol_F=1e-10, tol_R=1e-7, max_iter=2000)
    kw.update(minimize_kwargs or {})
    K = Functional(cell).K          # the NL kernel depends on nbar, L and T only

    def fn(pos, rho_prev):
        c = replace(cell, pos=np.asarray(pos, dtype=float))
        F = Functional(c, kernel=K)
        psi0 = None if rho_prev is None else np.sqrt(np.maximum(rho_prev, 0.0))
        r = lbfgs(F, psi0=psi0, **kw)
        if not r.converged:
            raise RuntimeError("electronic minimisation did not converge")
        return r.energies["total"], forces(c, r.rho), r.rho
    return fn

"""Direct minimisation of the free energy over sqrt(n) at fixed N_e.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper minimises the OFDFT free energy ("SCF iterations", Methods, Table 2
caption) without naming the optimiser.  Reading used here: L-BFGS (memory m,
two-loop recursion) on an unconstrained psi with n = N_e psi^2 / int psi^2, so
N_e is fixed exactly, and a strong-Wolfe line search (sufficient decrease c1,
curvature c2, cubic interpolation in the zoom phase).  Inner products are
int a b = dV sum a b.  Initial state: the uniform density.

Convergence: |dF| / N_ion below tol_F for 3 consecutive iterations and the
Euler-Lagrange residual R = (int n (v - mu)^2 / N_e)^(1/2) below tol_R.

Optional preconditioning (precond_c = c): the two-loop recursion starts from
H0 = gamma P instead of gamma I, with P f = IFFT[c / h(G) f~],
h(G) = c + G^2/2 (the vW kinetic operator shifted by c); the first direction
is -P g.  Two optional terms model more of the psi-Hessian at the mean
density: precond_k = f_K adds f_K 4 a^2 nbar^(2a-1) K(G) (the nonlocal
kernel's curvature), precond_h = f_H adds f_H 8 pi nbar / G^2 (a density wave
2 sqrt(nbar) dpsi against the Hartree energy) for G != 0; h is kept above
c / 1000.  Any symmetric positive-definite H0 leaves the minimum unchanged;
the tests check that the forms reach the same one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MinResult:
    psi: np.ndarray
    rho: np.ndarray
    energies: dict
    iterations: int
    evaluations: int
    converged: bool
    history: list = field(default_factory=list)


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic through (a, fa, ga), (b, fb, gb); None if none."""
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if disc < 0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = gb - ga + 2.0 * d2
    if den == 0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def line_search(phi, phi0, dphi0, t0, c1=1e-4, c2=0.9, max_evals=30):
    """Strong-Wolfe line search.  phi(t) -> (value, slope, payload).

    Returns (t, value, slope, payload) of the accepted point, or None.
    A point whose value change is below roundoff (|value - phi0| <= 1e-14
    |phi0|) is judged on the slope alone.
    """
    eps_f = 1e-14 * max(1.0, abs(phi0))

    def armijo_ok(t, f):
        return f <= phi0 + c1 * t * dphi0 or abs(f - phi0) <= eps_f

    def curv_ok(g):
        return abs(g) <= -c2 * dphi0

    evals = 0
    t_prev, f_prev, g_prev = 0.0, phi0, dphi0
    t = t0
    lo = hi = None
    while evals < max_evals:
        f, g, pay = phi(t)
        evals += 1
        if not armijo_ok(t, f) or (evals > 1 and f >= f_prev and abs(f - f_prev) > eps_f):
            lo, hi = (t_prev, f_prev, g_prev), (t, f, g)
            break
        if curv_ok(g):
            return t, f, g, pay
        if g >= 0:
            lo, hi = (t, f, g), (t_prev, f_prev, g_prev)
            lo_pay = pay
            break
        t_prev, f_prev, g_prev = t, f, g
        t = 2.0 * t
    else:
        return None
    # zoom between lo (satisfies Armijo, lower value) and hi
    while evals < max_evals:
        (a, fa, ga), (b, fb, gb) = lo, hi
        tc = _cubic_min(a, fa, ga, b, fb, gb)
        left, right = min(a, b), max(a, b)
        width = right - left
        if tc is None or not (left + 0.1 * width <= tc <= right - 0.1 * width):
            tc = 0.5 * (a + b)
        f, g, pay = phi(tc)
        evals += 1
        if not armijo_ok(tc, f) or (f >= fa and abs(f - fa) > eps_f):
            hi = (tc, f, g)
        else:
            if curv_ok(g):
                return tc, f, g, pay
            if g * (b - a) >= 0:
                hi = lo
            lo = (tc, f, g)
        if abs(hi[0] - lo[0]) < 1e-16 * max(1.0, abs(lo[0])):
            break
    return None


def lbfgs(functional, psi0=None, m=8, c1=1e-4, c2=0.9, tol_F=1e-6, tol_R=1e-4,
          max_iter=1000, verbose=False, precond_c=None, precond_k=0.0, precond_h=0.0) -> MinResult:
    """L-BFGS on psi (see module docstring).  functional.evaluate_psi(psi)
    returns (energies, gradient, rho)."""
    F = functional
    dV = F.dV
    if precond_c is None:
        P = lambda v: v
    else:
        from .functional import fft3, ifft3
        h = precond_c + 0.5 * F.G2
        if precond_k:
            h = h + precond_k * 4.0 * F.alpha ** 2 * F.nbar ** (2.0 * F.alpha - 1.0) * F.K
        if precond_h:
            with np.errstate(divide="ignore"):
                h = h + np.where(F.G2 > 0, precond_h * 8.0 * math.pi * F.nbar / np.where(F.G2 > 0, F.G2, 1.0), 0.0)
        pg = precond_c / np.maximum(h, 1e-3 * precond_c)
        P = lambda v: ifft3(fft3(v) * pg)
    n_ion = float(len(F.cell.Z))
    dot = lambda a, b: dV * float(np.sum(a * b))
    psi = np.full((F.n,) * 3, math.sqrt(F.nbar)) if psi0 is None else np.array(psi0, float)
    e, g, rho = F.evaluate_psi(psi)
    S, Y, RHO = [], [], []
    history = [dict(e)]
    small = 0
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        # two-loop recursion: d = -H g
        q = g.copy()
        alphas = []
        for s, y, r in zip(reversed(S), reversed(Y), reversed(RHO)):
            a = r * dot(s, q)
            alphas.append(a)
            q -= a * y
        z = P(q)
        if S:
            gamma = dot(S[-1], Y[-1]) / dot(Y[-1], Y[-1])
            t0 = 1.0
        else:
            gamma = 1.0
            t0 = 0.1 * math.sqrt(dot(psi, psi) / max(dot(z, z), 1e-300))
        z = gamma * z
        for (s, y, r), a in zip(zip(S, Y, RHO), reversed(alphas)):
            b = r * dot(y, z)
            z += (a - b) * s
        d = -z
        dphi0 = dot(g, d)
        if dphi0 >= 0:            # not a descent direction: restart from steepest descent
            S, Y, RHO = [], [], []
            d = -P(g)
            dphi0 = dot(g, d)
            t0 = 0.1 * math.sqrt(dot(psi, psi) / max(dot(d, d), 1e-300))

        def phi(t):
            x = psi + t * d
            ee, gg, rr = F.evaluate_psi(x)
            return ee["total"], dot(gg, d), (x, ee, gg, rr)

        res = line_search(phi, e["total"], dphi0, t0, c1=c1, c2=c2)
        if res is None:
            if verbose:
                print(f"line search failed at iteration {it}")
            break
        t, fnew, _, (xnew, enew, gnew, rnew) = res
        s = xnew - psi
        y = gnew - g
        sy = dot(s, y)
        if sy > 1e-300:
            S.append(s); Y.append(y); RHO.append(1.0 / sy)
            if len(S) > m:
                S.pop(0); Y.pop(0); RHO.pop(0)
        dF = abs(fnew - e["total"]) / n_ion
        psi, e, g, rho = xnew, enew, gnew, rnew
        history.append(dict(e))
        small = small + 1 if dF < tol_F else 0
        if verbose:
            print(f"it {it:4d} F {e['total']:.12f} dF/ion {dF:.3e} R {e['residual']:.3e} t {t:.3e}")
        if small >= 3 and e["residual"] < tol_R:
            converged = True
            break
    return MinResult(psi=psi, rho=rho, energies=e, iterations=it, evaluations=F.n_evals,
                     converged=converged, history=history)

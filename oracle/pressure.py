"""Electronic pressure P = -dF/dOmega of a periodic cell at a given density.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper reports pressures of warm dense hydrogen (Results, Table 1 from
OFDFT molecular dynamics; Fig. 3, the electronic pressure of fcc hydrogen
versus temperature) but prints no stress formula.  Reading used here: the
derivative of the free energy under a homogeneous dilation of the cell,

    L -> lambda L,  R_I -> lambda R_I,  n(r) -> n(r / lambda) / lambda^3,

at fixed temperature T and electron number, P = -(1 / (3 Omega)) dF/dlambda
at lambda = 1.  At a minimum of F over n this is the derivative of the
minimised free energy (to first order the path of n does not matter), i.e.
the pressure at fixed fractional ion coordinates, ion-ion term included; the
ideal-gas pressure N_i T_ion / Omega of moving ions is not part of it.

Term by term (f~ = FFT(f) / N as in oracle.cell, sums over the full grid):

* local functionals of n (finite-T TF at fixed T, LDA xc):
  F(lambda) = lambda^3 int f(n / lambda^3), so P = (1/Omega) int (n v - f);
  for TF, n v - f is the ideal-gas pressure n T p.
* vW is homogeneous of degree -2 in length: P = 2 E_vW / (3 Omega).
* Hartree and the Ewald ion-ion energy are of degree -1: P = E / (3 Omega).
* local pseudopotential: E_loc = sum_G Re[n~* S_Z] v~(G) with n~ -> n~/lambda^3
  and G -> G/lambda, so P = (1/3) sum_G Re[n~* V_loc] c(G),
  c = 1 - G^2 rc^2 / 2 for G != 0 (from v~ = -4 pi exp(-G^2 rc^2/4)/G^2) and
  c = 3 at G = 0 (the constant pi rc^2).
* NL: E_NL = Omega sum_G K(|G|; nbar) |w~|^2, w = n^a, and under the dilation
  E(lambda) = lambda^(3 - 6a) Omega sum_G K(|G|/lambda; nbar/lambda^3) |w~|^2, so
  P = -(1/3) sum_G |w~|^2 [(3 - 6a) K + dK], dK = d/dlambda K(|G|/lambda;
  nbar/lambda^3) at lambda = 1.  The kernel has no closed form (a Lindhard
  integral); dK is the Richardson extrapolation of central differences with
  steps 2e-3 and 1e-3 (error O(step^4)).
"""
from __future__ import annotations

import math

import numpy as np

from . import fermi_dirac as fd
from . import xc as xcmod
from .cell import m2_grid
from .functional import Functional, fft3, N_MIN, TERMS, ALPHA_DEFAULT
from .lindhard import kernel_table

DK_STEP = 2e-3


def kernel_dilation_derivative(m2_values, L: float, nbar: float, T: float, alpha: float,
                               step: float = DK_STEP) -> np.ndarray:
    """dK/dlambda of K(q/lambda; nbar/lambda^3) at lambda = 1 on integer shells."""
    def central(h):
        kp = kernel_table(m2_values, L * (1.0 + h), nbar / (1.0 + h) ** 3, T, alpha)
        km = kernel_table(m2_values, L * (1.0 - h), nbar / (1.0 - h) ** 3, T, alpha)
        return (kp - km) / (2.0 * h)
    return (4.0 * central(0.5 * step) - central(step)) / 3.0


def pressure(cell, rho, terms=TERMS, alpha=ALPHA_DEFAULT) -> dict:
    """Per-term pressure contributions and their total (hartree / bohr^3)."""
    F = Functional(cell, terms=terms, alpha=alpha)
    rho = np.asarray(rho, dtype=float)
    e, _ = F.evaluate(rho)
    Om, dV, T = F.Omega, F.dV, F.T
    nf = np.maximum(rho, N_MIN)
    p = {k: 0.0 for k in ("tf", "vw", "nl", "hartree", "loc", "xc", "ion")}
    if "tf" in F.terms:
        f, vt, _ = fd.tf_free_energy_density(nf, T)
        p["tf"] = dV * float(np.sum(nf * vt - f)) / Om
    if "xc" in F.terms:
        exc, vxc = xcmod.lda_xc(nf)
        p["xc"] = dV * float(np.sum(rho * (vxc - exc))) / Om
    p["vw"] = 2.0 * e["vw"] / (3.0 * Om)
    p["hartree"] = e["hartree"] / (3.0 * Om)
    p["ion"] = e["ion"] / (3.0 * Om)
    if "loc" in F.terms:
        c = np.where(F.G2 > 0, 1.0 - 0.5 * F.G2 * cell.rc ** 2, 3.0)
        p["loc"] = float(np.sum((np.conj(fft3(rho)) * F.Vloc).real * c)) / 3.0
    if "nl" in F.terms:
        m2 = m2_grid(F.n)
        u, inv = np.unique(m2, return_inverse=True)
        dK = kernel_dilation_derivative(u, F.L, F.nbar, T, F.alpha)[inv].reshape(m2.shape)
        w2 = np.abs(fft3(nf ** F.alpha)) ** 2
        p["nl"] = -float(np.sum(w2 * ((3.0 - 6.0 * F.alpha) * F.K + dK))) / 3.0
    p["total"] = sum(p[k] for k in ("tf", "vw", "nl", "hartree", "loc", "xc", "ion"))
    return p

"""The whole functional's minimum in a weak external potential eps cos(G0.r):
by the kernel's construction (Eq. 2) the second variation of TF + vW + NL at
nbar is -1/chi0(q;T), the finite-T Lindhard function; Hartree adds 4 pi/q^2
and the LDA adds f_xc = dv_xc/dn.  So the minimising density's amplitude at
G0 is

    A = -eps / (-1/chi0(q;T) + 4 pi/q^2 + f_xc)  + O(eps^2),

the static response of the interacting gas in this approximation.  This pins
the minimiser and every term of the functional together (a dropped Hartree
term, a wrong vW factor or XC sign moves A by tens of percent)."""
import math

import numpy as np

from oracle.functional import Functional, fft3
from oracle.minimize import lbfgs
from oracle.lindhard import chi0, mean_density_params
from oracle.xc import lda_xc
from workloads import fcc_cell


def test_minimum_responds_to_a_weak_cosine_as_the_interacting_gas():
    c = fcc_cell(n=16)
    F = Functional(c)
    n, L, T = c.n, c.L, c.T
    nbar = c.n_electrons / c.volume
    q = 2.0 * math.pi / L
    _, mu0, _ = mean_density_params(nbar, T)
    h = 1e-6 * nbar
    fxc = (lda_xc(np.array([nbar + h]))[1][0] - lda_xc(np.array([nbar - h]))[1][0]) / (2 * h)
    stiffness = -1.0 / chi0(q, mu0, T, nbar) + 4.0 * math.pi / q ** 2 + fxc
    dev = []
    for eps in (1e-3, 2e-3):
        # replace the ions' potential by eps cos(2 pi x / L): V(+-G0) = eps/2
        F.Vloc = np.zeros((n, n, n), complex)
        F.Vloc[1, 0, 0] = F.Vloc[n - 1, 0, 0] = eps / 2
        r = lbfgs(F, tol_F=1e-13, tol_R=1e-11, max_iter=3000)
        assert r.converged
        nt = fft3(r.rho)
        A = 2.0 * nt[1, 0, 0].real
        assert abs(nt[1, 0, 0].imag) < 1e-15 and abs(nt[0, 1, 0]) < 1e-15 and abs(nt[0, 0, 1]) < 1e-15
        dev.append(A / (-eps / stiffness) - 1.0)
    assert abs(dev[0]) < 1e-6
    assert 3.0 < dev[1] / dev[0] < 5.0          # the remainder is second order in eps

"""A special case of the variational minimum with a closed form: without the
gradient, nonlocal and Hartree terms the functional is local, so its minimum
at fixed N_e satisfies the Euler-Lagrange equation point by point,

    T eta(r) [+ v_xc(n(r))] + v_loc(r) = mu,   n(r) = sqrt2/pi^2 T^(3/2) I_{1/2}(eta(r)),

with mu fixed by the electron count (Eq. 1 with the Methods' local
pseudopotential and LDA).  Solving that equation per grid point by bisection
pins the oracle's minimiser, its projected gradient and the signs and factors
of the TF and XC potentials, independently of the line search and of the
transforms of n."""
import math

import numpy as np
import pytest

from oracle.functional import Functional, ifft3
from oracle.minimize import lbfgs
from oracle.fermi_dirac import fd_integral
from oracle.xc import lda_xc
from workloads import fcc_cell


def _density_of_eta(eta, T):
    return math.sqrt(2.0) / math.pi ** 2 * T ** 1.5 * np.asarray(fd_integral(0.5, eta.ravel())).reshape(eta.shape)


def _pointwise_minimum(v_loc, T, n_electrons, dV, with_xc):
    def n_of_mu(mu):
        if not with_xc:
            return _density_of_eta((mu - v_loc) / T, T)
        lo = np.full(v_loc.shape, -60.0)
        hi = np.full(v_loc.shape, 200.0)
        for _ in range(80):                       # T eta + v_xc(n(eta)) rises with eta here
            mid = 0.5 * (lo + hi)
            res = T * mid + lda_xc(_density_of_eta(mid, T))[1] - (mu - v_loc)
            hi = np.where(res > 0, mid, hi)
            lo = np.where(res > 0, lo, mid)
        return _density_of_eta(0.5 * (lo + hi), T)

    a, b = float(v_loc.min()) - 60 * T - 5.0, float(v_loc.max()) + 60 * T + 5.0
    for _ in range(90):                           # the electron count rises with mu
        mu = 0.5 * (a + b)
        if dV * n_of_mu(mu).sum() > n_electrons:
            b = mu
        else:
            a = mu
    return n_of_mu(0.5 * (a + b))


@pytest.mark.parametrize("terms", [("tf", "loc"), ("tf", "loc", "xc")])
def test_local_functional_minimum_solves_the_pointwise_equation(terms):
    c = fcc_cell(n=12)
    F = Functional(c, terms=terms)
    r = lbfgs(F, tol_F=1e-12, tol_R=1e-10, max_iter=3000)
    assert r.converged
    v_loc = ifft3(F.Vloc)
    ref = _pointwise_minimum(v_loc, c.T, c.n_electrons, F.dV, with_xc="xc" in terms)
    assert abs(F.dV * ref.sum() - c.n_electrons) < 1e-10 * c.n_electrons
    assert np.linalg.norm(r.rho - ref) / np.linalg.norm(ref) < 1e-8
    assert np.max(np.abs(r.rho - ref) / ref) < 1e-7
    # the density follows the attraction of the ions: a non-increasing function of v_loc
    order = np.argsort(v_loc.ravel(), kind="stable")
    steps = np.diff(r.rho.ravel()[order])
    assert np.all(steps <= 1e-7 * r.rho.max())

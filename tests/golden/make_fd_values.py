"""Writes fd_values.txt: complete Fermi-Dirac integrals
I_nu(eta) = int_0^inf x^nu / (1 + exp(x - eta)) dx = -Gamma(nu+1) Li_{nu+1}(-e^eta)
from mpmath's polylogarithm at 30 digits, a library independent of the
oracle's quadrature and of the CUDA path.

Run from the repository root:  python tests/golden/make_fd_values.py
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
POINTS = [(nu, eta) for nu in (0.5, 1.5, -0.5) for eta in (0.0, 5.0, -5.0)]
HEADER = """# Complete Fermi-Dirac integrals I_nu(eta) = int_0^inf x^nu / (1 + exp(x - eta)) dx
# (no 1/Gamma normalisation), the ingredient of the finite-T Thomas-Fermi
# functional F_s^TF of Eq. 1.  Values: I_nu(eta) = -Gamma(nu+1) Li_{nu+1}(-e^eta)
# evaluated with mpmath at 30 digits (independent of the oracle's quadrature).
# nu      eta      I_nu
"""


def values():
    import mpmath
    mpmath.mp.dps = 30
    out = []
    for nu, eta in POINTS:
        v = -mpmath.gamma(nu + 1) * mpmath.polylog(nu + 1, -mpmath.e ** mpmath.mpf(eta))
        out.append((nu, eta, mpmath.nstr(mpmath.re(v), 30)))   # real for real eta
    return out


def main():
    with open(os.path.join(HERE, "fd_values.txt"), "w") as f:
        f.write(HEADER)
        for nu, eta, v in values():
            f.write(f"{nu:<8} {eta:<8} {v}\n")


if __name__ == "__main__":
    main()

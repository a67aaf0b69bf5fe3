"""Generates fd_fit_tables.h: piecewise Chebyshev fits for the inverse
Fermi-Dirac integral and the Thomas-Fermi free-energy function.

For y = I_{1/2}(eta) (the reduced density pi^2 n / (sqrt2 T^(3/2)) of the
finite-T Thomas-Fermi term F_s^TF of Eq. 1) and s = ln y, the CUDA kernels
need
    eta(s)                              (v_TF = T eta)
    p(s) = (2/3) I_{3/2}(eta(s)) / y    (f_TF = sqrt2/pi^2 T^(5/2) y (eta - p))
Both are smooth in s.  On [S_LO, S_HI) they are tabulated as Chebyshev series
on equal intervals (an FP64 table of degree D64 on width W64 and an FP32 table
of degree D32 on width W32); outside, the kernels use the leading terms of the
non-degenerate series (s < S_LO) and of the Sommerfeld expansion (s >= S_HI).

Reference values: I_nu(eta) = -Gamma(nu+1) Li_{nu+1}(-e^eta) by mpmath for
eta <= 40, and the Sommerfeld series (exact to far below double precision for
half-integer nu at eta > 40, where the exponentially small part vanishes).
This generator is part of the library build tooling; it does not use the
test oracle.  Run: python gen_fd_fits.py  (writes fd_fit_tables.h beside it).
"""
from __future__ import annotations

import os
import sys

import mpmath as mp

mp.mp.dps = 34

S_LO, S_HI = -32.0, 24.0
W64, D64 = 0.5, 15
W32, D32 = 1.0, 7


def fd_int(nu, eta):
    nu = mp.mpf(nu)
    eta = mp.mpf(eta)
    if eta <= 40:
        return -mp.gamma(nu + 1) * mp.re(mp.polylog(nu + 1, -mp.exp(eta)))
    tot = mp.mpf(1)
    for k in range(1, 10):
        c = 2 * (1 - mp.mpf(2) ** (1 - 2 * k)) * mp.zeta(2 * k)
        c *= mp.gamma(nu + 2) / mp.gamma(nu + 2 - 2 * k)
        tot += c * eta ** (-2 * k)
    return eta ** (nu + 1) / (nu + 1) * tot


def eta_of_s(s):
    y = mp.exp(mp.mpf(s))
    u = y / mp.gamma(mp.mpf(1.5))
    if y < 1:
        guess = mp.log(u) + u / mp.sqrt(8)
    else:
        guess = (mp.mpf(1.5) * y) ** (mp.mpf(2) / 3)
    f = lambda e: mp.log(fd_int(0.5, e)) - mp.mpf(s)
    return mp.findroot(f, guess, tol=mp.mpf(10) ** (-30))


def funcs(s):
    e = eta_of_s(s)
    y = mp.exp(mp.mpf(s))
    p = mp.mpf(2) / 3 * fd_int(1.5, e) / y
    return e, p


def cheb_fit(f_nodes, deg):
    n = deg + 1
    coeffs = []
    for k in range(n):
        acc = mp.mpf(0)
        for j in range(n):
            x = mp.cos(mp.pi * (j + mp.mpf(0.5)) / n)
            acc += f_nodes[j] * mp.chebyt(k, x)
        c = 2 * acc / n
        if k == 0:
            c /= 2
        coeffs.append(c)
    return coeffs


def clenshaw(c, x):
    b1 = b2 = mp.mpf(0)
    for ck in reversed(c[1:]):
        b1, b2 = ck + 2 * x * b1 - b2, b1
    return c[0] + x * b1 - b2


def build_table(width, deg):
    nint = int(round((S_HI - S_LO) / width))
    ce, cp = [], []
    worst_e = worst_p = mp.mpf(0)
    for i in range(nint):
        a = mp.mpf(S_LO) + i * mp.mpf(width)
        mid = a + mp.mpf(width) / 2
        half = mp.mpf(width) / 2
        ev, pv = [], []
        for j in range(deg + 1):
            x = mp.cos(mp.pi * (j + mp.mpf(0.5)) / (deg + 1))
            e, p = funcs(mid + half * x)
            ev.append(e)
            pv.append(p)
        c1 = cheb_fit(ev, deg)
        c2 = cheb_fit(pv, deg)
        # check at interior points between the nodes
        for x in (mp.mpf(-0.97), mp.mpf(-0.41), mp.mpf(0.13), mp.mpf(0.77)):
            e, p = funcs(mid + half * x)
            worst_e = max(worst_e, abs(clenshaw(c1, x) - e) / max(1, abs(e)))
            worst_p = max(worst_p, abs(clenshaw(c2, x) - p) / max(1, abs(p)))
        ce.append(c1)
        cp.append(c2)
        sys.stderr.write(f"\r  width {width} interval {i + 1}/{nint}")
    sys.stderr.write(f"\n  max rel err eta {float(worst_e):.3e}  p {float(worst_p):.3e}\n")
    return nint, ce, cp, float(worst_e), float(worst_p)


def fmt(v, single):
    return (f"{float(v):.9e}f" if single else f"{float(v):.17e}")


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fd_fit_tables.h")
    n64, e64, p64, ee64, ep64 = build_table(W64, D64)
    n32, e32, p32, ee32, ep32 = build_table(W32, D32)
    lines = [
        "/* Generated by gen_fd_fits.py -- do not edit.",
        " * Piecewise Chebyshev series in s = ln y for eta(s) = I_{1/2}^{-1}(e^s) and",
        " * p(s) = (2/3) I_{3/2}(eta(s)) / e^s on [FD_S_LO, FD_S_HI).",
        f" * FP64 table: {n64} intervals of width {W64}, degree {D64}; max rel err eta {ee64:.2e}, p {ep64:.2e}.",
        f" * FP32 table: {n32} intervals of width {W32}, degree {D32}; max rel err eta {ee32:.2e}, p {ep32:.2e}.",
        " */",
        "#pragma once",
        f"#define FD_S_LO ({S_LO})",
        f"#define FD_S_HI ({S_HI})",
        f"#define FD64_W ({W64})",
        f"#define FD64_NINT {n64}",
        f"#define FD64_NC {D64 + 1}",
        f"#define FD32_W ({W32}f)",
        f"#define FD32_NINT {n32}",
        f"#define FD32_NC {D32 + 1}",
        f"#define FD64_MAX_REL_ERR_ETA ({ee64:.3e})",
        f"#define FD32_MAX_REL_ERR_ETA ({ee32:.3e})",
    ]

    def arr(name, tab, single, typ):
        lines.append(f"static __device__ __align__(16) const {typ} {name}[{len(tab)}][{len(tab[0])}] = {{")
        for row in tab:
            lines.append("  {" + ", ".join(fmt(v, single) for v in row) + "},")
        lines.append("};")

    arr("fd64_eta", e64, False, "double")
    arr("fd64_p", p64, False, "double")
    arr("fd32_eta", e32, True, "float")
    arr("fd32_p", p32, True, "float")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()

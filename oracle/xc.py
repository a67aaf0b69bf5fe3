"""Perdew-Zunger (1981) LDA exchange-correlation, spin-unpolarised.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper treats exchange-correlation with the Perdew-Zunger LDA in the
adiabatic (ground-state) approximation (Methods, "Numerical calculations for
OFDFT and KSDFT").  The paper prints no formula; this is the textbook PZ81
parametrisation of the Ceperley-Alder correlation energy:

  r_s = (3 / (4 pi n))^(1/3)
  e_x = -(3/4) (3/pi)^(1/3) n^(1/3)                         v_x = (4/3) e_x
  e_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)           (r_s >= 1)
  e_c = A ln r_s + B + C r_s ln r_s + D r_s                 (r_s <  1)
  v_c = e_c - (r_s / 3) d e_c / d r_s

PZ81 fixes B and D of the high-density branch by requiring e_c and
d e_c / d r_s to be continuous at r_s = 1, where the two branches meet.  The
published three-digit values (B = -0.048, D = -0.0116) are the rounding of
that solution and leave a step of 3.2e-5 Ha in e_c (2.8e-5 Ha in v_c) at
r_s = 1, which no minimiser can settle across: a density that straddles
r_s = 1 (hydrogen at r_s = 1) stalls with its residual stuck near 3e-4 Ha.
Reading used here: B and D are solved from the two continuity conditions
given gamma, beta1, beta2, A and C (they differ from the printed values by
1.9e-5 and 1.3e-5).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA, BETA1, BETA2 = -0.1423, 1.0529, 0.3334
A, C = 0.0311, 0.0020
# continuity at r_s = 1:  B + D = gamma / (1 + beta1 + beta2)  and
# A + C + D = -gamma (beta1/2 + beta2) / (1 + beta1 + beta2)^2
_DEN1 = 1.0 + BETA1 + BETA2
D = -GAMMA * (0.5 * BETA1 + BETA2) / _DEN1 ** 2 - A - C
B = GAMMA / _DEN1 - D
CX = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)


def rs_of_n(n):
    return (3.0 / (4.0 * math.pi * np.asarray(n, dtype=float))) ** (1.0 / 3.0)


def exchange(n):
    """(e_x, v_x) per electron."""
    n = np.asarray(n, dtype=float)
    ex = -CX * np.cbrt(n)
    return ex, 4.0 / 3.0 * ex


def correlation(n):
    """(e_c, v_c) per electron."""
    rs = rs_of_n(n)
    hi = rs >= 1.0
    rs_h = np.where(hi, rs, 1.0)
    sq = np.sqrt(rs_h)
    den = 1.0 + BETA1 * sq + BETA2 * rs_h
    ec_h = GAMMA / den
    # d e_c / d r_s on the r_s >= 1 branch
    dec_h = -GAMMA * (0.5 * BETA1 / sq + BETA2) / den ** 2
    rs_l = np.where(hi, 1.0, rs)
    ln = np.log(rs_l)
    ec_l = A * ln + B + C * rs_l * ln + D * rs_l
    dec_l = A / rs_l + C * ln + C + D
    ec = np.where(hi, ec_h, ec_l)
    dec = np.where(hi, dec_h, dec_l)
    vc = ec - rs / 3.0 * dec
    return ec, vc


def lda_xc(n):
    """(e_xc per electron, v_xc) for the PZ81 LDA."""
    ex, vx = exchange(n)
    ec, vc = correlation(n)
    return ex + ec, vx + vc

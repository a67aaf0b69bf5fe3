"""Plain FP64 CPU oracle for the finite-temperature orbital-free DFT hot path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
restatement of what the method computes, used to check the CUDA library.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and the two share no
code (inputs come from the separate ``workloads`` package).

Modules (each function cites the part of the paper, or the textbook definition
the paper names, that it follows):

* ``fermi_dirac``  Fermi-Dirac integrals, their inverse, the finite-T
                   Thomas-Fermi free energy (F_s^TF of Eq. 1).
* ``fdint.c``,     the quadrature behind ``fermi_dirac`` in plain C
  ``_native``      (panels of 20-point Gauss-Legendre in t with x = t^2),
                   compiled with the host gcc into oracle/_build/.
* ``xc``           Perdew-Zunger LDA exchange-correlation (Methods).
* ``lindhard``     finite-T Lindhard response and the F_0^NL kernel (Eq. 2).
* ``cell``         grid, G vectors, structure factor, local pseudopotential,
                   Ewald ion-ion energy.
* ``functional``   F_s[n;T] = TF + vW + NL (Eq. 1) plus Hartree, local PP and
                   XC; energy and potential.
* ``minimize``     L-BFGS on sqrt(n) at fixed electron number.
* ``sei``          electron-ion and ion-ion static structure factors on |q|
                   shells, and the direct-sum form for large cells (Methods,
                   static structure factors; a trajectory average is the mean
                   of the per-snapshot values).
* ``forces``       Hellmann-Feynman forces on the ions (Methods, molecular
                   dynamics).
* ``pressure``     P = -dF/dOmega under a homogeneous dilation (Results,
                   Table 1 and Fig. 3 report pressures).
* ``md``           Born-Oppenheimer ion dynamics, velocity Verlet with a
                   Nose-Hoover thermostat (Methods, molecular dynamics).

Parity status: every function is pinned by the tests in ``tests/test_oracle_*``
against closed forms, library routines or brute force, except the end-to-end
physics against the paper's figures, which needs data the paper does not print
(parity unpinned for that comparison only).
"""

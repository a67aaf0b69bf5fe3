"""The Python binding refuses arguments the kernels would read or write out
of bounds (wrong size, type, layout or device) before any library call; run
on CPU with a plan shell that has no library behind it."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2601_23002_gb300.api import Plan


class _NoLib:
    def __getattr__(self, name):
        def call(*a, **k):
            raise AssertionError(f"library call {name} reached with a bad argument")
        return call


def _shell(n=8, n_ion=4, dtype=torch.float64):
    p = Plan.__new__(Plan)
    p.lib = _NoLib()
    p._Z = np.ones(n_ion)
    p.n = n
    p.dtype = dtype
    p.device = 0
    p.stream = None
    p._p = ctypes.c_void_p()
    return p


@pytest.mark.parametrize("pos", [np.zeros((3, 3)), np.zeros(13), np.zeros((4, 2))])
def test_host_positions_must_hold_n_ion_by_3_values(pos):
    with pytest.raises(ValueError, match="positions"):
        _shell().structure_factor(pos)


def test_fields_must_match_the_plan():
    p = _shell()
    for t in (torch.zeros(8 ** 3, dtype=torch.float64),                     # host memory
              torch.zeros(7 ** 3, dtype=torch.float64),
              torch.zeros(8 ** 3, dtype=torch.float32)):
        with pytest.raises(ValueError, match="8\\^3 elements"):
            p._field(t, "rho")
    for call in (p.energy_potential, p.forces, p.pressure, p.sei_shells):
        with pytest.raises(ValueError):
            call(torch.zeros(8 ** 3, dtype=torch.float64))
    with pytest.raises(ValueError):
        p.minimize(torch.zeros(8 ** 3, dtype=torch.float64))

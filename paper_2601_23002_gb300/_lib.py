"""ctypes view of include/ofdft.h.  Raises if the CUDA library is missing."""
from __future__ import annotations

import ctypes
import os

from .build import LIB

c_double_p = ctypes.POINTER(ctypes.c_double)

OFDFT_OK = 0
OFDFT_ERR_INVALID = 1
OFDFT_ERR_CUDA = 2
OFDFT_ERR_OOM = 3
OFDFT_ERR_NOT_CONVERGED = 4
OFDFT_ERR_TIMEOUT = 5
OFDFT_ERR_NAN = 6
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "TIMEOUT", 6: "NAN"}

OFDFT_FP64 = 0
OFDFT_FP32 = 1
TERM_TF, TERM_VW, TERM_NL, TERM_XC, TERM_HARTREE, TERM_LOC = 1, 2, 4, 8, 16, 32
TERMS_ALL = 63


class Cell(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("n", ctypes.c_int), ("n_ion", ctypes.c_int),
                ("Z", c_double_p), ("rc", ctypes.c_double), ("T", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("terms", ctypes.c_int), ("alpha", ctypes.c_double),
                ("fd64", ctypes.c_int)]


class Energies(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("F_TF", "E_vW", "E_NL", "E_H", "E_loc", "E_xc", "E_ion", "F_total", "N_e", "mu",
                 "residual")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MinOpts(ctypes.Structure):
    _fields_ = [("tol_F_per_ion", ctypes.c_double), ("tol_residual", ctypes.c_double),
                ("m", ctypes.c_int), ("max_iter", ctypes.c_int), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("e", Energies), ("iterations", ctypes.c_int), ("evaluations", ctypes.c_int),
                ("status", ctypes.c_int)]


class MdOpts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("T_ion", ctypes.c_double), ("tau", ctypes.c_double),
                ("n_shells", ctypes.c_int), ("min", MinOpts)]


class MdThermostat(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("s", ctypes.c_double), ("steps_done", ctypes.c_int)]


class MdFrame(ctypes.Structure):
    _fields_ = [("e_pot", ctypes.c_double), ("kinetic", ctypes.c_double), ("conserved", ctypes.c_double),
                ("xi", ctypes.c_double), ("evaluations", ctypes.c_int), ("iterations", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


EXPORTS = ["ofdft_default_opts", "ofdft_default_min_opts", "ofdft_last_error", "ofdft_version",
           "ofdft_plan_create", "ofdft_plan_destroy", "ofdft_plan_bytes", "ofdft_structure_factor",
           "ofdft_energy_potential", "ofdft_minimize", "ofdft_sei_shells",
           "ofdft_profile_enable", "ofdft_profile_read", "ofdft_sei_shells_static",
           "ofdft_minimize_batch", "ofdft_autotune", "ofdft_set_tiles", "ofdft_forces",
           "ofdft_pressure", "ofdft_md_run", "ofdft_energy_potential_async"]

_lib = None


def load(path: str | None = None):
    """Load libofdft_gb300.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        from .build import build
        build()
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.ofdft_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.ofdft_default_opts.restype = None
    L.ofdft_default_min_opts.argtypes = [ctypes.POINTER(MinOpts)]
    L.ofdft_default_min_opts.restype = None
    L.ofdft_last_error.restype = ctypes.c_char_p
    L.ofdft_version.restype = ctypes.c_char_p
    L.ofdft_plan_create.argtypes = [ctypes.POINTER(Cell), ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.ofdft_plan_create.restype = ctypes.c_int
    L.ofdft_plan_destroy.argtypes = [vp]
    L.ofdft_plan_destroy.restype = None
    L.ofdft_plan_bytes.argtypes = [ctypes.POINTER(Cell), ctypes.POINTER(Opts)]
    L.ofdft_plan_bytes.restype = ctypes.c_size_t
    L.ofdft_structure_factor.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.ofdft_structure_factor.restype = ctypes.c_int
    L.ofdft_energy_potential.argtypes = [vp, vp, vp, ctypes.POINTER(Energies), vp]
    L.ofdft_energy_potential.restype = ctypes.c_int
    L.ofdft_minimize.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(MinOpts), ctypes.POINTER(Result), vp]
    L.ofdft_minimize.restype = ctypes.c_int
    L.ofdft_sei_shells.argtypes = [vp, vp, ctypes.c_int, c_double_p, c_double_p, vp]
    L.ofdft_sei_shells.restype = ctypes.c_int
    L.ofdft_forces.argtypes = [vp, vp, c_double_p, vp]
    L.ofdft_forces.restype = ctypes.c_int
    L.ofdft_pressure.argtypes = [vp, vp, c_double_p, vp]
    L.ofdft_pressure.restype = ctypes.c_int
    L.ofdft_energy_potential_async.argtypes = [vp, vp, vp, vp, vp]
    L.ofdft_energy_potential_async.restype = ctypes.c_int
    L.ofdft_md_run.argtypes = [vp, vp, ctypes.c_int, c_double_p, c_double_p, c_double_p,
                               ctypes.POINTER(MdOpts), ctypes.POINTER(MdThermostat), ctypes.c_int,
                               ctypes.POINTER(MdFrame), c_double_p, c_double_p, c_double_p, vp]
    L.ofdft_md_run.restype = ctypes.c_int
    L.ofdft_sei_shells_static.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_int, vp, vp, vp]
    L.ofdft_sei_shells_static.restype = ctypes.c_int
    L.ofdft_minimize_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(MinOpts), ctypes.POINTER(Result), ctypes.c_int]
    L.ofdft_minimize_batch.restype = ctypes.c_int
    L.ofdft_autotune.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.ofdft_autotune.restype = ctypes.c_int
    L.ofdft_set_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.ofdft_set_tiles.restype = ctypes.c_int
    L.ofdft_profile_enable.argtypes = [vp, ctypes.c_int]
    L.ofdft_profile_enable.restype = ctypes.c_int
    L.ofdft_profile_read.argtypes = [vp, ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.ofdft_profile_read.restype = ctypes.c_int
    _lib = L
    return L


def last_error() -> str:
    return load().ofdft_last_error().decode()

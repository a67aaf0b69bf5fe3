"""The CUDA library builds, loads and exports every entry point that
include/ofdft.h declares; host-side validation rejects bad input without a
GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    with open(os.path.join(ROOT, "include", "ofdft.h")) as f:
        txt = f.read()
    for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ofdft_\w+)\s*\(", txt, re.M):
        names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_23002_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(lib, nm), nm


def test_binding_covers_declared_symbols():
    from paper_2601_23002_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.EXPORTS) | {"ofdft_default_opts"}


def test_defaults(lib):
    from paper_2601_23002_gb300 import _lib as C
    o = C.Opts()
    lib.ofdft_default_opts(ctypes.byref(o))
    assert o.precision == C.OFDFT_FP64 and o.terms == C.TERMS_ALL and o.alpha == 0.5
    m = C.MinOpts()
    lib.ofdft_default_min_opts(ctypes.byref(m))
    assert m.m == 8 and m.tol_F_per_ion == 1e-6 and m.c1 == 1e-4 and m.c2 == 0.9
    assert b"sm_103a" in lib.ofdft_version()


def _cell(C, n=32, Z=(3.0, 3.0), L=7.6, T=0.2, rc=1.0):
    Za = np.array(Z, dtype=np.float64)
    return C.Cell(L, n, len(Za), Za.ctypes.data_as(C.c_double_p), rc, T), Za


def test_plan_bytes_and_validation(lib):
    from paper_2601_23002_gb300 import _lib as C
    o = C.Opts(C.OFDFT_FP32, C.TERMS_ALL, 0.5)
    cell, keep = _cell(C)
    b = lib.ofdft_plan_bytes(ctypes.byref(cell), ctypes.byref(o))
    assert b > 20 * 32 ** 3 * 4
    for bad in (dict(n=33), dict(n=14), dict(L=-1.0), dict(T=0.0), dict(Z=(3.0, -1.0)), dict(n=1024),
                dict(rc=float("inf")), dict(rc=float("nan")), dict(T=float("nan")), dict(L=float("inf"))):
        kw = dict(n=32, Z=(3.0, 3.0), L=7.6, T=0.2)
        kw.update(bad)
        c2, keep2 = _cell(C, **kw)
        assert lib.ofdft_plan_bytes(ctypes.byref(c2), ctypes.byref(o)) == 0
        p = ctypes.c_void_p()
        rc = lib.ofdft_plan_create(ctypes.byref(c2), ctypes.byref(o), None, ctypes.byref(p))
        assert rc == C.OFDFT_ERR_INVALID and not p.value
        assert len(lib.ofdft_last_error()) > 0
    o_bad = C.Opts(7, C.TERMS_ALL, 0.5)
    p = ctypes.c_void_p()
    assert lib.ofdft_plan_create(ctypes.byref(cell), ctypes.byref(o_bad), None, ctypes.byref(p)) == C.OFDFT_ERR_INVALID
    o_bad = C.Opts(C.OFDFT_FP64, C.TERMS_ALL, 1.5)
    assert lib.ofdft_plan_create(ctypes.byref(cell), ctypes.byref(o_bad), None, ctypes.byref(p)) == C.OFDFT_ERR_INVALID


def test_null_arguments_rejected(lib):
    from paper_2601_23002_gb300 import _lib as C
    assert lib.ofdft_energy_potential(None, None, None, None, None) == C.OFDFT_ERR_INVALID
    assert lib.ofdft_minimize(None, None, 1, None, None, None) == C.OFDFT_ERR_INVALID
    assert lib.ofdft_structure_factor(None, None, 0, None, None) == C.OFDFT_ERR_INVALID
    lib.ofdft_plan_destroy(None)


def test_fft_factorisations_cover_workload_grids():
    # every 2,3,5-smooth grid 8..512, odd or even, factors into the supported radices
    from workloads.cells import _is_smooth
    from paper_2601_23002_gb300 import _lib as C
    lib = C.load()
    o = C.Opts(C.OFDFT_FP64, C.TERMS_ALL, 0.5)
    for n in range(8, 513):
        if _is_smooth(n):
            cell, keep = _cell(C, n=n)
            assert lib.ofdft_plan_bytes(ctypes.byref(cell), ctypes.byref(o)) > 0, n


def test_minimiser_options_checked_alike_by_every_entry_point(lib):
    # the options are checked before anything touches a plan or the GPU
    from paper_2601_23002_gb300 import _lib as C
    good = C.MinOpts(1e-6, 1e-4, 8, 100, 1e-4, 0.9)
    bads = [C.MinOpts(1e-6, 1e-4, 0, 100, 1e-4, 0.9), C.MinOpts(1e-6, 1e-4, 9, 100, 1e-4, 0.9),
            C.MinOpts(1e-6, 1e-4, 8, 0, 1e-4, 0.9), C.MinOpts(1e-6, 1e-4, 8, 100, 0.5, 0.4),
            C.MinOpts(1e-6, 1e-4, 8, 100, 1e-4, 1.0), C.MinOpts(float("nan"), 1e-4, 8, 100, 1e-4, 0.9),
            C.MinOpts(1e-6, -1.0, 8, 100, 1e-4, 0.9)]
    for o in bads:
        assert lib.ofdft_minimize(None, None, 1, ctypes.byref(o), None, None) == C.OFDFT_ERR_INVALID
        assert "minimiser options" in C.last_error()
        assert lib.ofdft_minimize_batch(None, None, 0, 1, ctypes.byref(o), None, 1) == C.OFDFT_ERR_INVALID
    # valid options: the NULL plan is what fails; an empty batch has nothing to do
    assert lib.ofdft_minimize(None, None, 1, ctypes.byref(good), None, None) == C.OFDFT_ERR_INVALID
    assert "NULL" in C.last_error()
    assert lib.ofdft_minimize_batch(None, None, 0, 1, ctypes.byref(good), None, 1) == C.OFDFT_OK
    # zero tolerances are allowed (never met: the minimiser runs to max_iter)
    zero = C.MinOpts(0.0, 0.0, 8, 100, 1e-4, 0.9)
    assert lib.ofdft_minimize_batch(None, None, 0, 1, ctypes.byref(zero), None, 1) == C.OFDFT_OK


C_CONSUMER = r"""
#include <stdio.h>
#include <string.h>
#include "ofdft.h"

int main(void) {
    ofdft_opts o;
    ofdft_default_opts(&o);
    ofdft_min_opts m;
    ofdft_default_min_opts(&m);
    const double Z[2] = {3.0, 3.0};
    ofdft_cell c = {.L = 7.6, .n = 32, .n_ion = 2, .Z = Z, .rc = 1.0, .T = 0.2};
    size_t b = ofdft_plan_bytes(&c, &o);
    c.n = 33;
    size_t bad = ofdft_plan_bytes(&c, &o);
    int rc = ofdft_minimize(NULL, NULL, 1, &m, NULL, NULL);
    printf("%s|%zu|%zu|%d|%d|%s\n", ofdft_version(), b, bad, rc, m.m, ofdft_last_error());
    return (b > 0 && bad == 0 && rc == OFDFT_ERR_INVALID) ? 0 : 1;
}
"""


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    # the boundary is a C ABI: a C99 program includes the header, links the
    # shared library and calls its host-side entry points (no GPU needed)
    import shutil
    import subprocess
    from paper_2601_23002_gb300 import _lib
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    _lib.load()                                        # builds the library if needed
    so = _lib.LIB
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                         so, "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, (run.stdout, run.stderr)
    version, b, bad, rc, m, err = run.stdout.strip().split("|")
    assert int(b) > 0 and int(bad) == 0 and int(m) == 8 and "NULL" in err

"""The allocation-free S_ei entry point (ofdft_sei_shells_static) agrees with
the plan-based ofdft_sei_shells on the same density and ions, on two calls in
a row with different grids (so nothing left in its fixed scratch array from
one call leaks into the next), and refuses requests beyond its fixed size.

It exists for callers that cannot allocate device memory while they run; this
file is collected last so that a stop-at-first-failure run has already run
every other test."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2601_23002_gb300 as og
from paper_2601_23002_gb300 import _lib
from workloads import random_cell, SEED_BASE


def _density(cell, seed):
    rng = np.random.default_rng(seed)
    n = cell.n
    x = np.arange(n) / n
    f = np.zeros((n, n, n))
    for k in rng.integers(-3, 4, size=(5, 3)):
        f += np.cos(2 * math.pi * (k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :])
                    + rng.uniform(0, 6.28))
    rho = np.exp(0.3 * f)
    return rho * cell.n_electrons / (rho.sum() * cell.volume / rho.size)


def _static_call(lib, rho_d, pos_d, cell, n_shells):
    q = torch.full((n_shells,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.full((n_shells,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.ofdft_sei_shells_static(ctypes.c_void_p(rho_d.data_ptr()), ctypes.c_void_p(pos_d.data_ptr()),
                                     cell.n_ion, cell.L, cell.n, cell.n_electrons, n_shells,
                                     ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.last_error()
    return q.cpu().numpy(), s.cpu().numpy()


def test_static_sei_matches_plan_entry_point_on_two_calls():
    lib = _lib.load()
    cells = [random_cell(SEED_BASE + 41, 12, 1.0, 2.0, 1.0, 48), random_cell(SEED_BASE + 42, 7, 3.0, 1.8, 0.5, 32)]
    for i, cell in enumerate(cells):
        rho = torch.tensor(_density(cell, 10 + i), dtype=torch.float64, device="cuda")
        pos = torch.tensor(cell.pos, dtype=torch.float64, device="cuda")
        plan = og.plan_for_cell(cell)
        q_ref, s_ref = plan.sei_shells(rho, 120)
        plan.close()
        q, s = _static_call(lib, rho, pos, cell, 120)
        assert np.allclose(q, q_ref, rtol=1e-14, atol=0)
        assert np.max(np.abs(s - s_ref)) < 1e-10


def test_static_sei_rejects_requests_beyond_its_fixed_size():
    lib = _lib.load()
    cell = random_cell(SEED_BASE + 43, 5, 1.0, 2.0, 1.0, 96)
    rho = torch.ones(96 ** 3, dtype=torch.float64, device="cuda")
    pos = torch.tensor(cell.pos, dtype=torch.float64, device="cuda")
    out = torch.zeros(300, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.ofdft_sei_shells_static(p(rho), p(pos), 5, cell.L, 96, 5.0, 10, p(out), p(out), st) == _lib.OFDFT_ERR_INVALID
    assert "64" in _lib.last_error()
    small = torch.ones(32 ** 3, dtype=torch.float64, device="cuda")
    assert lib.ofdft_sei_shells_static(p(small), p(pos), 5, cell.L, 32, 5.0, 300, p(out), p(out), st) == _lib.OFDFT_ERR_INVALID


def test_static_sei_concurrent_calls_give_the_sequential_results():
    """Two host threads, each on its own stream, call the entry point on
    different grids at the same time; the per-device lock keeps them off each
    other's scratch, so every result equals the one-at-a-time result."""
    import threading
    lib = _lib.load()
    cells = [random_cell(SEED_BASE + 44, 12, 1.0, 2.0, 1.0, 48), random_cell(SEED_BASE + 45, 9, 1.0, 1.6, 0.8, 32)]
    rhos = [torch.tensor(_density(c, 20 + i), dtype=torch.float64, device="cuda") for i, c in enumerate(cells)]
    poss = [torch.tensor(c.pos, dtype=torch.float64, device="cuda") for c in cells]
    ref = [_static_call(lib, r, p, c, 100) for c, r, p in zip(cells, rhos, poss)]
    out = [[], []]
    errors = []

    def worker(k):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for _ in range(6):
                    out[k].append(_static_call(lib, rhos[k], poss[k], cells[k], 100))
        except Exception as e:          # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k in (0, 1):
        assert len(out[k]) == 6
        for q, s in out[k]:
            assert np.array_equal(q, ref[k][0]) and np.array_equal(s, ref[k][1])


def test_static_sei_at_its_largest_grid_and_shell_count():
    """n = 64 with 256 shells, the sizes the fixed array was laid out for: the
    shells' half-spectrum entries (counted here on the host) stay within the
    array's 16384 slots, and the result equals the plan entry point's."""
    h = 32
    m2s = sorted({mx * mx + my * my + mz * mz for mx in range(-h, h) for my in range(-h, h)
                  for mz in range(h + 1)} - {0})[:256]
    want = set(m2s)
    entries = sum(1 for mx in range(-h, h) for my in range(-h, h) for mz in range(h + 1)
                  if mx * mx + my * my + mz * mz in want)
    assert entries <= 16384
    lib = _lib.load()
    cell = random_cell(SEED_BASE + 46, 20, 1.0, 2.2, 0.7, 64)
    rho = torch.tensor(_density(cell, 30), dtype=torch.float64, device="cuda")
    pos = torch.tensor(cell.pos, dtype=torch.float64, device="cuda")
    plan = og.plan_for_cell(cell)
    q_ref, s_ref = plan.sei_shells(rho, 256)
    plan.close()
    for _ in range(2):
        q, s = _static_call(lib, rho, pos, cell, 256)
        assert np.allclose(q, q_ref, rtol=1e-14, atol=0)
        assert np.max(np.abs(s - s_ref)) < 1e-10

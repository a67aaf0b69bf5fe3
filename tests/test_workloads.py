"""The seeded synthetic inputs follow their stated recipe: grid sizes the
smallest 2,3,5-smooth n (odd or even) within their clamp, ions at least 0.8 bohr apart under the
minimum image, cell sides from r_s, temperatures from theta, MD velocities
without net momentum, and the same draws on every call."""
import math

import numpy as np
import pytest

from workloads import batch_cells, config_cell, random_cell, SEED_BASE
from workloads.cells import smooth_grid, _is_smooth, serving_requests, md_velocities, hydrogen_md_cells, \
    PROTON_MASS

HARTREE_EV = 27.211386245988


def _min_image_distance(pos, L):
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    r[np.diag_indices(len(pos))] = np.inf
    return r.min()


def test_grid_rule():
    for L in np.linspace(5.0, 40.0, 57):
        n = smooth_grid(L, 0.25, 48, 96)
        assert 48 <= n <= 96 and _is_smooth(n)
        if n < 96:
            assert n >= L / 0.25 - 1e-9
            # the smallest such size
            assert all(not _is_smooth(k) for k in range(max(48, math.ceil(L / 0.25 - 1e-9)), n))
    # the sizes the batched workload's clamp allows, odd ones included
    sizes = {smooth_grid(L, 0.25, 48, 96) for L in np.linspace(11.0, 24.5, 2000)}
    assert sizes == {48, 50, 54, 60, 64, 72, 75, 80, 81, 90, 96}


def test_batched_snapshots_follow_the_recipe():
    cells = batch_cells(64)
    for c in cells:
        assert 16 <= c.n_ion <= 128 and len(set(c.Z)) == 1 and c.Z[0] in (1.0, 3.0, 4.0)
        rs = (3.0 * c.volume / (4.0 * math.pi * c.n_electrons)) ** (1.0 / 3.0)
        assert abs(rs - c.meta["rs"]) < 1e-12 and 1.0 <= rs <= 3.0 and 0.1 <= c.theta <= 2.0
        assert np.all((c.pos >= 0) & (c.pos < c.L))
        assert _min_image_distance(c.pos, c.L) >= 0.8
    again = batch_cells(64)
    assert all(np.array_equal(a.pos, b.pos) and a.n == b.n for a, b in zip(cells, again))


def test_bench_cell_temperature_is_the_papers_12_5_eV():
    # 64 H at r_s = 2, theta = 1: T = theta (3 pi^2 nbar)^(2/3) / 2; the paper
    # quotes 12.5 eV for hydrogen at r_s = 2 and theta = 1 (Methods, Table 2)
    c = config_cell(2)
    rs = (3.0 * c.volume / (4.0 * math.pi * c.n_electrons)) ** (1.0 / 3.0)
    assert abs(rs - 2.0) < 1e-12 and c.n == 128 and c.n_ion == 64
    assert abs(c.T * HARTREE_EV - 12.5) < 0.05
    assert _min_image_distance(c.pos, c.L) >= 0.8


def test_serving_stream_is_seeded_and_sized():
    t1, c1 = serving_requests(40)
    t2, c2 = serving_requests(40)
    assert np.array_equal(t1, t2) and all(np.array_equal(a.pos, b.pos) for a, b in zip(c1, c2))
    assert np.all(np.diff(t1) > 0)
    for c in c1:
        assert 8 <= c.n_ion <= 512 and 32 <= c.n <= 160 and _is_smooth(c.n)


def test_md_inputs():
    cells = hydrogen_md_cells()
    assert [c.n_ion for c in cells] == [32, 14, 14]
    for c in cells:
        mass = np.full(c.n_ion, PROTON_MASS)
        v = md_velocities(SEED_BASE + 7, mass, c.T)
        assert np.allclose((mass[:, None] * v).sum(0), 0.0, atol=1e-12)
        assert np.array_equal(v, md_velocities(SEED_BASE + 7, mass, c.T))
        # the MD cells keep a hard core of 0.6 r_s, scaled with the density
        assert _min_image_distance(c.pos, c.L) >= 0.6 * c.meta["rs"] and _is_smooth(c.n)
        assert c.n >= c.L / (0.10 / 0.529177210903) - 1e-9        # 0.10 Angstrom or finer

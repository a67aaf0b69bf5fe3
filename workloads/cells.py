"""Synthetic cells with the shapes of the paper's workloads.

The paper simulates hydrogen and beryllium cells of 14 to 1024 ions at
r_s = 1 to 3.23 and theta = 0.1 to 4 on real-space grids of 0.035 to 0.10
Angstrom spacing (Results; Methods, "Numerical calculations" and "Molecular
dynamics").  The five workloads below keep those shapes: cubic boxes, seeded
random ion positions with a hard-core rejection, one ion species per cell and
grid spacings of 0.1 to 0.25 bohr.

Units are Hartree atomic units.  The temperature is carried both as the reduced
degeneracy theta = T / T_F (how a workload is specified) and as T in Hartree,
with T_F = (3 pi^2 nbar)^(2/3) / 2 and nbar = N_e / Omega.  That conversion is
the definition of theta, not part of the functional.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2601230020


@dataclass
class Cell:
    """One periodic cubic cell with point ions and a real-space grid."""
    L: float                 # cell side (bohr)
    n: int                   # grid points per side
    Z: np.ndarray            # valence charge per ion, shape [n_ion]
    pos: np.ndarray          # Cartesian ion positions (bohr), shape [n_ion, 3]
    theta: float             # T / T_F
    rc: float = 1.0          # Gaussian smoothing radius of the local pseudopotential (bohr)
    label: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_ion(self) -> int:
        return int(len(self.Z))

    @property
    def volume(self) -> float:
        return self.L ** 3

    @property
    def n_electrons(self) -> float:
        return float(np.sum(self.Z))

    @property
    def T(self) -> float:
        """Electron temperature in Hartree from theta = T / T_F."""
        nbar = self.n_electrons / self.volume
        return self.theta * 0.5 * (3.0 * math.pi ** 2 * nbar) ** (2.0 / 3.0)


def _is_smooth(k: int) -> bool:
    for p in (2, 3, 5):
        while k % p == 0:
            k //= p
    return k == 1


def smooth_grid(L: float, spacing: float, lo: int, hi: int) -> int:
    """Smallest 2,3,5-smooth n >= L/spacing (odd or even), clamped to [lo, hi]."""
    target = max(lo, int(math.ceil(L / spacing - 1e-9)))
    k = target
    while not _is_smooth(k):
        k += 1
    return int(min(k, hi))


def _random_positions(rng: np.random.Generator, n_ion: int, L: float,
                      min_sep: float) -> np.ndarray:
    """Uniform positions in [0, L)^3, rejecting any draw closer than min_sep
    (minimum image) to an ion already placed."""
    pos = np.zeros((n_ion, 3))
    placed = 0
    tries = 0
    while placed < n_ion:
        p = rng.uniform(0.0, L, size=3)
        tries += 1
        if tries > 1000000:
            raise RuntimeError("could not place ions at this density")
        if placed:
            d = pos[:placed] - p
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep ** 2:
                continue
        pos[placed] = p
        placed += 1
    return pos


def fcc_cell(a: float = 7.6, Z: float = 3.0, n: int = 32, theta: float = 0.5,
             rc: float = 1.0) -> Cell:
    """Conventional 4-ion fcc cell of side a (the 32^3 plain-FP64 workload)."""
    frac = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], float)
    return Cell(L=a, n=n, Z=np.full(4, float(Z)), pos=frac * a, theta=theta, rc=rc,
                label=f"fcc4_Z{Z:g}_n{n}")


def small_fcc_cell(n: int = 16, theta: float = 0.5) -> Cell:
    """The fcc workload on a coarser grid, for fast oracle tests."""
    c = fcc_cell(n=n, theta=theta)
    c.label = f"fcc4_Z3_n{n}"
    return c


def random_cell(seed: int, n_ion: int, Z: float, rs: float, theta: float, n: int,
                min_sep: float = 0.8, rc: float = 1.0, label: str = "") -> Cell:
    """n_ion ions of charge Z at seeded random positions; box from r_s."""
    ne = n_ion * Z
    L = (ne * 4.0 * math.pi * rs ** 3 / 3.0) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    pos = _random_positions(rng, n_ion, L, min_sep)
    return Cell(L=L, n=n, Z=np.full(n_ion, float(Z)), pos=pos, theta=theta, rc=rc,
                label=label or f"rand{n_ion}_Z{Z:g}_rs{rs:.3g}_n{n}",
                meta={"seed": seed, "rs": rs})


def config_cell(index: int) -> Cell:
    """The single-cell workloads: 1 = fcc 32^3, 2 = 64 H at r_s=2 on 128^3,
    4 = 1024 Z=3 ions at r_s=2.5 on 256^3."""
    if index == 1:
        return fcc_cell()
    if index == 2:
        return random_cell(SEED_BASE + 2 * 1000, 64, 1.0, 2.0, 1.0, 128,
                           label="rand64_H_rs2_n128")
    if index == 4:
        return random_cell(SEED_BASE + 4 * 1000, 1024, 3.0, 2.5, 0.3, 256,
                           label="rand1024_Z3_rs2.5_n256")
    raise ValueError(f"no single-cell workload {index}")


def batch_cells(count: int = 64, spacing: float = 0.25, lo: int = 48,
                hi: int = 96, cfg: int = 3) -> list[Cell]:
    """Independent snapshots of uneven size: 16-128 ions, Z in {1,3,4},
    r_s ~ U[1,3], theta ~ U[0.1,2], grid from ~0.25 bohr spacing."""
    out = []
    for i in range(count):
        seed = SEED_BASE + cfg * 1000 + i
        rng = np.random.default_rng(seed)
        n_ion = int(rng.integers(16, 129))
        Z = float(rng.choice([1.0, 3.0, 4.0]))
        rs = float(rng.uniform(1.0, 3.0))
        theta = float(rng.uniform(0.1, 2.0))
        ne = n_ion * Z
        L = (ne * 4.0 * math.pi * rs ** 3 / 3.0) ** (1.0 / 3.0)
        n = smooth_grid(L, spacing, lo, hi)
        pos = _random_positions(rng, n_ion, L, 0.8)
        out.append(Cell(L=L, n=n, Z=np.full(n_ion, Z), pos=pos, theta=theta,
                        label=f"b{i}_N{n_ion}_Z{Z:g}_n{n}",
                        meta={"seed": seed, "rs": rs}))
    return out


def serving_requests(count: int = 2000, spacing: float = 0.25, lo: int = 32,
                     hi: int = 160, rate: float = 1.0, cfg: int = 5):
    """Poisson stream of cells: N_ion log-uniform in [8,512], Z in {1,3,4},
    r_s ~ U[1,3], theta ~ U[0.1,2]; returns (arrival_times, cells)."""
    rng = np.random.default_rng(SEED_BASE + cfg * 1000)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    cells = []
    for i in range(count):
        r = np.random.default_rng(SEED_BASE + cfg * 1000 + 1 + i)
        n_ion = int(round(math.exp(r.uniform(math.log(8), math.log(512)))))
        Z = float(r.choice([1.0, 3.0, 4.0]))
        rs = float(r.uniform(1.0, 3.0))
        theta = float(r.uniform(0.1, 2.0))
        ne = n_ion * Z
        L = (ne * 4.0 * math.pi * rs ** 3 / 3.0) ** (1.0 / 3.0)
        n = smooth_grid(L, spacing, lo, hi)
        pos = _random_positions(r, n_ion, L, 0.8)
        cells.append(Cell(L=L, n=n, Z=np.full(n_ion, Z), pos=pos, theta=theta,
                          label=f"r{i}_N{n_ion}_Z{Z:g}_n{n}", meta={"rs": rs}))
    return arrivals, cells


PROTON_MASS = 1836.15267343          # electron masses (CODATA 2018)
BOHR_PER_ANGSTROM = 1.0 / 0.529177210903


def md_velocities(seed: int, mass, T_ion: float) -> np.ndarray:
    """Seeded Maxwell-Boltzmann velocities [n_ion, 3] at temperature T_ion
    (Ha, atomic units), with the total momentum removed."""
    mass = np.asarray(mass, dtype=float)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(len(mass), 3)) * np.sqrt(T_ion / mass)[:, None]
    p = (mass[:, None] * v).sum(axis=0)
    return v - p / mass.sum()


def hydrogen_md_cells() -> list[Cell]:
    """The three warm-dense-hydrogen MD systems whose time per MD step the
    paper tabulates (Methods, Table 2): 32 H at r_s = 1, 14 H at r_s = 2 and
    14 H at r_s = 3.23, all at theta = 1, on a 0.10 Angstrom grid (rounded up
    to a 2,3,5-smooth size), seeded random liquid-like positions."""
    out = []
    for i, (n_ion, rs) in enumerate(((32, 1.0), (14, 2.0), (14, 3.23))):
        L = (n_ion * 4.0 * math.pi * rs ** 3 / 3.0) ** (1.0 / 3.0)
        n = smooth_grid(L, 0.10 * BOHR_PER_ANGSTROM, 8, 512)
        out.append(random_cell(SEED_BASE + 5000 + i, n_ion, 1.0, rs, 1.0, n, min_sep=0.6 * rs,
                               label=f"md_H{n_ion}_rs{rs:g}_n{n}"))
    return out

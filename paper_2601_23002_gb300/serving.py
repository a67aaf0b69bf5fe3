"""Continuous-batching request loop for density optimisations of mixed sizes.

Requests (a cell each) arrive over time.  A request is admitted as soon as a
worker slot is free and the device has room for its plan
(`ofdft_plan_bytes` against free HBM minus a reserve and minus what admitted
but not yet allocated requests will take).  Each slot owns a CUDA stream and
runs plan creation (kernel table), structure factor and L-BFGS for its
request; the calls release the GIL, so the slots' work overlaps on the GPU and
a request that arrives while others are running starts without waiting for
them to finish.  A request's density, spectra and kernel table stay resident
on the device from admission until its result is copied out.

All numerics run in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import Plan, OfdftError


@dataclass
class Request:
    rid: int
    cell: object
    arrival: float                  # seconds after the start of the run
    admitted: float = -1.0
    finished: float = -1.0
    result: dict = field(default_factory=dict)
    density: np.ndarray | None = None
    error: str = ""
    nbytes: int = 0                 # device bytes of its plan

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def solve(cell, precision, tol, autotune=True, stream=None, device="cuda"):
    """One request: plan, structure factor, minimisation from the uniform
    density, plan freed.  An FP32 minimisation that stops above the
    tolerances (its line search lost in FP32 rounding, as on small cold
    cells close to the 1e-4 Ha residual) is finished by an FP64 plan started
    from the FP32 density; the result says so (`finished_fp64`).
    Returns (result, density)."""
    dt = torch.float32 if precision == "fp32" else torch.float64
    plan = Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc, precision=precision, stream=stream)
    try:
        plan.structure_factor(cell.pos)
        if autotune:
            plan.autotune()
        rho = torch.empty(cell.n ** 3, dtype=dt, device=device)
        out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=tol[0], tol_residual=tol[1])
    finally:
        plan.close()
    out["finished_fp64"] = False
    if precision == "fp32" and not out["converged"]:
        p64 = Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc, precision="fp64", stream=stream)
        try:
            p64.structure_factor(cell.pos)
            r64 = rho.double()
            o64 = p64.minimize(r64, start_uniform=False, tol_F_per_ion=tol[0], tol_residual=tol[1])
        finally:
            p64.close()
        o64["evaluations"] += out["evaluations"]
        o64["iterations"] += out["iterations"]
        o64["finished_fp64"] = True
        out, rho = o64, r64
    return out, rho


class Server:
    def __init__(self, slots: int = 8, precision: str = "fp32", reserve_bytes: int = 4 << 30,
                 tol_F_per_ion: float = 1e-6, tol_residual: float = 1e-4, keep_density: bool = False,
                 autotune: bool = True, device: int = 0):
        self.slots = slots
        self.precision = precision
        self.reserve = reserve_bytes
        self.tol = (tol_F_per_ion, tol_residual)
        self.keep_density = keep_density
        self.autotune = autotune
        self.device = device
        self._lock = threading.Condition()
        self._pending: list[Request] = []
        self._committed = 0          # bytes of admitted plans not yet released
        self._done: list[Request] = []
        self._stop = False

    # -------------------------------------------------------------- workers
    def _plan_bytes(self, cell) -> int:
        return Plan.plan_bytes(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc, precision=self.precision)

    def _serve_one(self, req: Request, stream) -> None:
        with torch.cuda.stream(stream):
            out, rho = solve(req.cell, self.precision, self.tol, self.autotune, stream,
                             torch.device("cuda", self.device))
            if self.keep_density:
                req.density = rho.double().cpu().numpy()
            else:
                stream.synchronize()
            req.result = out

    def _slot_stream(self):
        torch.cuda.set_device(self.device)
        return torch.cuda.Stream(device=self.device)

    def _free_bytes(self) -> int:
        return torch.cuda.mem_get_info(self.device)[0]

    def _worker(self) -> None:
        stream = self._slot_stream()
        while True:
            with self._lock:
                while not self._stop and not self._ready():
                    self._lock.wait(timeout=0.002)
                if self._stop and not self._pending:
                    return
                req = self._take()
                if req is None:
                    continue
            try:
                self._serve_one(req, stream)
            except OfdftError as e:
                req.error = str(e)
            except Exception as e:       # e.g. an allocation failure: the request fails, the slot lives on
                req.error = f"{type(e).__name__}: {e}"
            req.finished = time.perf_counter() - self._t0
            with self._lock:
                self._committed -= req.nbytes
                self._done.append(req)
                self._lock.notify_all()

    def _ready(self) -> bool:
        now = time.perf_counter() - self._t0
        return bool(self._pending) and self._pending[0].arrival <= now and self._fits(self._pending[0])

    def _fits(self, req: Request) -> bool:
        # admission by memory: the plans of every admitted, unfinished request
        # must fit in the device memory that was free at start minus a reserve
        return self._committed + req.nbytes <= self._budget

    def _take(self) -> Request | None:
        if not self._ready():
            return None
        req = self._pending.pop(0)
        req.admitted = time.perf_counter() - self._t0
        self._committed += req.nbytes
        return req

    def prepare(self, cells) -> dict:
        """Tune the FFT tile schedule once per grid size (outside any timed
        run); returns {n: tiles}."""
        tiles = {}
        for cell in cells:
            if cell.n in tiles:
                continue
            p = Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc, precision=self.precision)
            p.structure_factor(cell.pos)
            tiles[cell.n] = p.autotune()[0]
            p.close()
        torch.cuda.synchronize()
        return tiles

    # ------------------------------------------------------------------ run
    def run(self, arrivals, cells) -> list[Request]:
        """Serve cells[i] arriving at arrivals[i] seconds; returns the requests
        (with admission / finish times and results) in completion order."""
        reqs = [Request(i, c, float(a)) for i, (a, c) in enumerate(zip(arrivals, cells))]
        for r in reqs:
            r.nbytes = self._plan_bytes(r.cell)
        reqs.sort(key=lambda r: r.arrival)
        self._budget = self._free_bytes() - self.reserve
        if any(r.nbytes > self._budget for r in reqs):
            raise ValueError("a request does not fit in device memory even alone")
        self._pending = reqs
        self._done = []
        self._stop = False
        self._t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(self.slots)]
        for t in threads:
            t.start()
        with self._lock:
            while len(self._done) < len(reqs):
                self._lock.wait(timeout=0.01)
            self._stop = True
            self._lock.notify_all()
        for t in threads:
            t.join()
        self.wall = time.perf_counter() - self._t0
        return list(self._done)


def summarize(done: list[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in done if not r.error])
    ok = [r for r in done if not r.error and r.result.get("converged")]
    return {"requests": len(done), "converged": len(ok), "errors": sum(1 for r in done if r.error),
            "finished_fp64": sum(1 for r in done if r.result.get("finished_fp64")),
            "snapshots_per_s": len(ok) / wall if wall > 0 else 0.0,
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "wall_s": wall}


def run_sequential(cells, precision: str = "fp32", tol_F_per_ion: float = 1e-6, tol_residual: float = 1e-4,
                   keep_density: bool = False, autotune: bool = True):
    """The plain single-instance path: one request after another on one stream.
    Returns (results, seconds)."""
    out = []
    t0 = time.perf_counter()
    for cell in cells:
        r, rho = solve(cell, precision, (tol_F_per_ion, tol_residual), autotune)
        if keep_density:
            r["density"] = rho.double().cpu().numpy()
        torch.cuda.synchronize()
        out.append(r)
    return out, time.perf_counter() - t0

"""Thin Python binding over the C-ABI (argument marshalling only).

Every step of the computation runs in the CUDA library; PyTorch provides the
device memory and the stream.  Functions raise OfdftError on a non-zero
status (minimize returns the partial result with status NOT_CONVERGED).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as C


class OfdftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ofdft status {C.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(rc: int):
    if rc != C.OFDFT_OK:
        raise OfdftError(rc, C.last_error())


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """One cell: L (bohr), n, Z[n_ion], rc (bohr), T (Ha)."""

    def __init__(self, L: float, n: int, Z, T: float, rc: float = 1.0, precision: str = "fp64",
                 terms: int = C.TERMS_ALL, alpha: float = 0.5, stream=None, fd64: bool = False):
        self.lib = C.load()
        self._Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64))
        self.cell = C.Cell(float(L), int(n), int(self._Z.size),
                           self._Z.ctypes.data_as(C.c_double_p), float(rc), float(T))
        self.opts = C.Opts(C.OFDFT_FP32 if precision == "fp32" else C.OFDFT_FP64, int(terms), float(alpha),
                           int(bool(fd64)))
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.n = int(n)
        self.stream = stream
        self._p = ctypes.c_void_p()
        _check(self.lib.ofdft_plan_create(ctypes.byref(self.cell), ctypes.byref(self.opts),
                                          _stream_ptr(stream), ctypes.byref(self._p)))
        self.device = torch.cuda.current_device()     # the plan's memory lives here

    @staticmethod
    def plan_bytes(L, n, Z, T, rc=1.0, precision="fp64", terms=C.TERMS_ALL, alpha=0.5) -> int:
        lib = C.load()
        Zc = np.ascontiguousarray(np.asarray(Z, dtype=np.float64))
        cell = C.Cell(float(L), int(n), int(Zc.size), Zc.ctypes.data_as(C.c_double_p), float(rc), float(T))
        opts = C.Opts(C.OFDFT_FP32 if precision == "fp32" else C.OFDFT_FP64, int(terms), float(alpha))
        return int(lib.ofdft_plan_bytes(ctypes.byref(cell), ctypes.byref(opts)))

    def close(self):
        if self._p:
            self.lib.ofdft_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _on_device(self, t: torch.Tensor) -> bool:
        return t.is_cuda and t.device.index == self.device

    def _field(self, t: torch.Tensor, name: str):
        # the kernels read and write exactly n^3 elements of the plan's type on
        # the plan's device: anything else is refused here, before any launch
        n = self.n
        if not (self._on_device(t) and t.dtype == self.dtype and t.is_contiguous() and t.numel() == n ** 3):
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor with {n}^3 elements "
                             f"on cuda:{self.device}")
        return ctypes.c_void_p(t.data_ptr())

    def structure_factor(self, pos, S_out: torch.Tensor | None = None):
        ni = self._Z.size
        if isinstance(pos, torch.Tensor) and pos.is_cuda:
            if not (self._on_device(pos) and pos.numel() == 3 * ni):
                raise ValueError(f"pos must hold {ni} x 3 positions on cuda:{self.device}")
            p = pos.contiguous().to(torch.float64)
            self._pos_keep = p
            ptr, dev = ctypes.c_void_p(p.data_ptr()), 1
        else:
            a = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
            if a.size != 3 * ni:
                raise ValueError(f"pos must hold {ni} x 3 positions, got {a.size} values")
            self._pos_keep = a
            ptr, dev = ctypes.c_void_p(a.ctypes.data), 0
        sptr = None
        if S_out is not None:
            nh = self.n // 2 + 1
            want = torch.complex64 if self.dtype == torch.float32 else torch.complex128
            if not (self._on_device(S_out) and S_out.dtype == want and S_out.is_contiguous()
                    and S_out.numel() == self.n * self.n * nh):
                raise ValueError("S_out must be a contiguous complex tensor [n, n, n/2+1] on the plan's device")
            sptr = ctypes.c_void_p(S_out.data_ptr())
        _check(self.lib.ofdft_structure_factor(self._p, ptr, dev, sptr, _stream_ptr(self.stream)))

    def energy_potential(self, rho: torch.Tensor, v_out: torch.Tensor | None = None) -> dict:
        e = C.Energies()
        vp = self._field(v_out, "v_out") if v_out is not None else None
        _check(self.lib.ofdft_energy_potential(self._p, self._field(rho, "rho"), vp, ctypes.byref(e),
                                               _stream_ptr(self.stream)))
        return e.as_dict()

    ENERGY_KEYS = ("F_TF", "E_vW", "E_NL", "E_H", "E_loc", "E_xc", "E_ion", "F_total", "N_e", "mu", "residual")

    def energy_potential_async(self, rho: torch.Tensor, v_out: torch.Tensor | None = None,
                               e_out: torch.Tensor | None = None) -> torch.Tensor:
        """Queue one evaluation (ofdft_energy_potential_async); returns the
        device tensor (float64 [11], order of ENERGY_KEYS) the energies are
        written to, without synchronising the stream."""
        if e_out is None:
            e_out = torch.empty(11, dtype=torch.float64, device=rho.device)
        if not (self._on_device(e_out) and e_out.dtype == torch.float64 and e_out.is_contiguous() and e_out.numel() >= 11):
            raise ValueError("e_out must be a contiguous CUDA float64 tensor with 11 elements")
        vp = self._field(v_out, "v_out") if v_out is not None else None
        _check(self.lib.ofdft_energy_potential_async(self._p, self._field(rho, "rho"), vp,
                                                     ctypes.c_void_p(e_out.data_ptr()), _stream_ptr(self.stream)))
        return e_out

    def minimize(self, rho: torch.Tensor, start_uniform: bool = True, tol_F_per_ion: float = 1e-6,
                 tol_residual: float = 1e-4, m: int = 8, max_iter: int = 1000, c1: float = 1e-4,
                 c2: float = 0.9, raise_on_fail: bool = False) -> dict:
        o = C.MinOpts(tol_F_per_ion, tol_residual, m, max_iter, c1, c2)
        r = C.Result()
        rc = self.lib.ofdft_minimize(self._p, self._field(rho, "rho"), int(bool(start_uniform)),
                                     ctypes.byref(o), ctypes.byref(r), _stream_ptr(self.stream))
        if rc not in (C.OFDFT_OK, C.OFDFT_ERR_NOT_CONVERGED) or (raise_on_fail and rc):
            _check(rc)
        out = r.e.as_dict()
        out.update(iterations=r.iterations, evaluations=r.evaluations, status=r.status,
                   converged=r.status == C.OFDFT_OK)
        return out

    def autotune(self):
        """Pick the FFT tile schedule (cached per grid size and precision)."""
        t = (ctypes.c_int * 3)()
        us = ctypes.c_double(0)
        _check(self.lib.ofdft_autotune(self._p, _stream_ptr(self.stream), t, ctypes.byref(us)))
        return tuple(t), us.value

    def set_tiles(self, tiles):
        t = (ctypes.c_int * 3)(*[int(x) for x in tiles])
        _check(self.lib.ofdft_set_tiles(self._p, t))

    def profile_enable(self, timing: bool = True):
        """Reset the per-kernel counters; with timing, bracket launches by events."""
        _check(self.lib.ofdft_profile_enable(self._p, int(bool(timing))))

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms, algorithmic bytes)} since the last enable."""
        cnt = ctypes.c_int(0)
        _check(self.lib.ofdft_profile_read(self._p, None, 0, ctypes.byref(cnt)))
        arr = (C.KernelStat * max(1, cnt.value))()
        _check(self.lib.ofdft_profile_read(self._p, arr, cnt.value, ctypes.byref(cnt)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms), float(arr[i].bytes))
                for i in range(cnt.value)}

    def sei_shells(self, rho: torch.Tensor, n_shells: int = 200):
        q = np.zeros(n_shells)
        s = np.zeros(n_shells)
        _check(self.lib.ofdft_sei_shells(self._p, self._field(rho, "rho"), int(n_shells),
                                         q.ctypes.data_as(C.c_double_p), s.ctypes.data_as(C.c_double_p),
                                         _stream_ptr(self.stream)))
        return q, s

    def forces(self, rho: torch.Tensor) -> np.ndarray:
        """Hellmann-Feynman forces [n_ion, 3] (hartree/bohr) at density rho for
        the positions of the last set_ions (ofdft_forces)."""
        f = np.zeros((self._Z.size, 3))
        _check(self.lib.ofdft_forces(self._p, self._field(rho, "rho"), f.ctypes.data_as(C.c_double_p),
                                     _stream_ptr(self.stream)))
        return f

    PRESSURE_TERMS = ("tf", "vw", "nl", "hartree", "loc", "xc", "ion", "total")

    def pressure(self, rho: torch.Tensor) -> dict:
        """Pressure -dF/dOmega (hartree/bohr^3) per term and total at density
        rho (ofdft_pressure)."""
        p = np.zeros(8)
        _check(self.lib.ofdft_pressure(self._p, self._field(rho, "rho"), p.ctypes.data_as(C.c_double_p),
                                       _stream_ptr(self.stream)))
        return dict(zip(self.PRESSURE_TERMS, p.tolist()))

    def md_run(self, rho: torch.Tensor, pos, vel, mass, n_steps: int, dt: float, T_ion: float = 0.0,
               tau: float = 0.0, thermostat=(0.0, 0.0), n_shells: int = 0, start_uniform: bool = False,
               tol_F_per_ion: float = 1e-6, tol_residual: float = 1e-4, m: int = 8, max_iter: int = 1000,
               c1: float = 1e-4, c2: float = 0.9) -> dict:
        """Ion dynamics (ofdft_md_run).  pos, vel: [n_ion, 3] (bohr, atomic
        units of velocity), mass: [n_ion] (electron masses); T_ion <= 0 runs
        NVE.  Returns the new pos, vel and thermostat (xi, s), per-step frames
        and, with n_shells > 0, the shells q and the per-call sums of S_ei and
        S_ii over the steps (divide by n_steps for trajectory averages)."""
        ni = self._Z.size
        x = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(ni, 3)).copy()
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64).reshape(ni, 3)).copy()
        ms = np.ascontiguousarray(np.asarray(mass, dtype=np.float64).reshape(ni))
        o = C.MdOpts(float(dt), float(T_ion), float(tau), int(n_shells),
                     C.MinOpts(tol_F_per_ion, tol_residual, m, max_iter, c1, c2))
        th = C.MdThermostat(float(thermostat[0]), float(thermostat[1]), 0)
        frames = (C.MdFrame * max(1, n_steps))()
        ns = max(1, int(n_shells))
        q, sei, sii = np.zeros(ns), np.zeros(ns), np.zeros(ns)
        dp = lambda a: a.ctypes.data_as(C.c_double_p)
        rc = self.lib.ofdft_md_run(self._p, self._field(rho, "rho"), int(bool(start_uniform)), dp(x), dp(v),
                                   dp(ms), ctypes.byref(o), ctypes.byref(th), int(n_steps), frames, dp(q),
                                   dp(sei), dp(sii), _stream_ptr(self.stream))
        out = dict(pos=x, vel=v, thermostat=(th.xi, th.s), steps_done=th.steps_done, status=rc,
                   frames={k: np.array([getattr(frames[i], k) for i in range(th.steps_done)])
                           for k, _ in C.MdFrame._fields_})
        if n_shells > 0:
            out.update(q=q, sei_sum=sei, sii_sum=sii)
        if rc != C.OFDFT_OK:
            _check(rc)
        return out


def minimize_batch(plans, rhos, concurrency: int = 8, start_uniform: bool = True, tol_F_per_ion: float = 1e-6,
                   tol_residual: float = 1e-4, m: int = 8, max_iter: int = 1000, c1: float = 1e-4,
                   c2: float = 0.9) -> list:
    """Minimise independent snapshots concurrently (ofdft_minimize_batch).
    Returns one result dict per plan, in order."""
    lib = C.load()
    cnt = len(plans)
    for p, r in zip(plans, rhos):
        p._field(r, "rho")
    P = (ctypes.c_void_p * cnt)(*[p._p.value for p in plans])
    R = (ctypes.c_void_p * cnt)(*[r.data_ptr() for r in rhos])
    res = (C.Result * cnt)()
    o = C.MinOpts(tol_F_per_ion, tol_residual, m, max_iter, c1, c2)
    torch.cuda.synchronize()
    rc = lib.ofdft_minimize_batch(P, R, cnt, int(bool(start_uniform)), ctypes.byref(o), res, int(concurrency))
    if rc not in (C.OFDFT_OK, C.OFDFT_ERR_NOT_CONVERGED):
        _check(rc)
    out = []
    for i in range(cnt):
        d = res[i].e.as_dict()
        d.update(iterations=res[i].iterations, evaluations=res[i].evaluations, status=res[i].status,
                 converged=res[i].status == C.OFDFT_OK)
        out.append(d)
    return out


def minimize(cell, rho: torch.Tensor | None = None, precision: str = "fp64", device="cuda", **opts):
    """One snapshot end to end: plan + structure factor for `cell` (a
    workloads.Cell or any object with L, n, Z, pos, rc, T), minimisation from
    `rho` (a density on the device) or from the uniform density, plan freed.
    Returns (converged density, result dict)."""
    plan = plan_for_cell(cell, precision=precision)
    try:
        dt = torch.float32 if precision == "fp32" else torch.float64
        out = torch.empty(cell.n ** 3, dtype=dt, device=device)
        if rho is not None:
            out.copy_(rho.reshape(-1))
        res = plan.minimize(out, start_uniform=rho is None, **opts)
    finally:
        plan.close()
    return out, res


def plan_for_cell(cell, precision="fp64", terms=C.TERMS_ALL, alpha=0.5, stream=None, fd64=False) -> Plan:
    """Plan + structure factor for a workloads.Cell (or any object with
    L, n, Z, pos, rc, T).  fd64: FP32 plans invert the Fermi-Dirac integral
    in FP64 (ofdft_opts.fd64)."""
    p = Plan(cell.L, cell.n, cell.Z, cell.T, rc=cell.rc, precision=precision, terms=terms, alpha=alpha,
             stream=stream, fd64=fd64)
    try:
        p.structure_factor(cell.pos)
    except BaseException:
        p.close()          # free the device memory now, not at garbage collection
        raise
    return p

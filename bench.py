#!/usr/bin/env python3
"""Benchmark of the OFDFT hot path on one GB300 (or N replicas under torchrun).

Metric: converged OFDFT snapshots/s at 1e-6 Ha/atom (with functional evals/s
and effective HBM GB/s alongside) on the largest single-GPU workload: 1024
ions of Z = 3 at seeded random positions with a 0.8 bohr hard core, r_s = 2.5
bohr, theta = 0.3, 256^3 grid, FP32 bulk arithmetic with FP64 sums and line
search.  A step is one snapshot end to end: structure factor, local
pseudopotential and Ewald energy (the per-snapshot setup), L-BFGS from the
uniform density to |dF|/ion < 1e-6 Ha for 3 iterations and residual < 1e-4
Ha, then the electron-ion structure factor S_ei on the first 200 |q| shells.
The nonlocal kernel table (fixed by nbar and T) is built at plan creation,
outside the timed region, as the paper excludes its kernel-table
initialisation from its timings.  The inputs (1.7 GB of plan state) exceed
the 126 MB L2; the L2 is flushed before every step all the same.

Alongside: the 64-H r_s = 2 theta = 1 128^3 cell (FP32 and the FP64 plain
path), the FP64 path on the 256^3 cell, the error of each against the
oracle's converged minimum, the batched form (64 snapshots of 48^3-96^3), the
serving form (2000 Poisson requests of 32^3-160^3) and MD time per step.

Arms:
  default           the CUDA library.
  --impl reference  the FP64 CPU oracle on the host cores, each step a bounded
                    sample of the same snapshot (per-snapshot setup on a
                    sample of the ions + one functional evaluation),
                    extrapolated to a snapshot with the oracle's own
                    evaluation count for this cell.
Under torchrun (N > 1) every rank solves its own copy of the snapshot stream
(replicas, no data-path collective); value = all ranks' snapshots / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged OFDFT snapshots/sec and functional evals/sec at 1e-6 Ha/atom; HBM GB/s"
WORKLOAD = ("1024 Z=3 ions, r_s=2.5 bohr, theta=0.3, 256^3 grid, seeded random positions (0.8 bohr hard "
            "core), Gaussian-smoothed Coulomb ions rc=1.0, L-BFGS m=8 from the uniform density to 1e-6 "
            "Ha/atom and residual 1e-4 Ha, then S_ei on 200 |q| shells")
HEADLINE_CFG = 4
N_SHELLS = 200
TOL_F, TOL_R = 1e-6, 1e-4


def config_dict(world: int, snaps: int, cell=None) -> dict:
    """The `config` object of both arms' JSON lines (same keys)."""
    workload = WORKLOAD if cell is None or cell.label == "rand1024_Z3_rs2.5_n256" else \
        f"{cell.label}: {cell.n_ion} ions, {cell.n}^3 grid, theta={cell.theta:g}, L-BFGS to 1e-6 Ha/atom, S_ei"
    return {"workload": workload, "global_batch": snaps, "seq_len": None, "parallelism": f"replicas x{world}",
            "l2": "flushed between steps (256 MB write outside the timed interval); the 256^3 cell's "
                  "1.7 GB plan state exceeds the L2 as well"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cell", type=int, default=HEADLINE_CFG, choices=[1, 2, 4],
                    help="single-cell workload of a step: 4 = 1024 Z=3 ions on 256^3 (the headline), "
                         "2 = 64 H on 128^3, 1 = the 4-ion fcc cell on 32^3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cfg2", action="store_true", help="skip the 128^3 single-cell block")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--serving", type=int, default=2000,
                    help="Poisson requests of the serving block (0 = skip)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-md", action="store_true", help="skip the MD time-per-step block")
    ap.add_argument("--tiles", default=None,
                    help="fixed FFT tile schedule 'rows,ycols,xcols' for the headline plan instead of the "
                         "autotuner's (for profiling runs, whose timings the profiler distorts)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def kernel_source_hash() -> str:
    """Hash of the sources that define the kernels and their launch shapes
    (api.cu holds only the C-ABI's host-side checks and dispatch)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2601_23002_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")) and f != "api.cu":
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples; OFDFT_CLOCKS_DIR keeps them somewhere chosen (default: the temp directory)
        d = os.environ.get("OFDFT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"ofdft_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        rows = [r for r in rows if len(r) >= 9]      # a partial last line when the sampler stopped
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:                        # "[N/A]" and the like
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        smx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smx) if smx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our arm
def flush_l2(buf):
    buf.add_(1.0)


def golden_minima():
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_minima.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def error_vs_oracle(cell, out, rho=None):
    """|F - F_oracle| / N_ion against the oracle's converged minimum of the
    same cell (tests/golden, written from oracle/ alone), and the relative L2
    distance of the density where the oracle's density is stored."""
    g = golden_minima().get(cell.label)
    if not g:
        return None
    r = {"dF_per_ion": abs(out["F_total"] - g["energies"]["total"]) / cell.n_ion,
         "oracle_tol_F_per_ion": g["tol_F_per_ion"], "oracle_tol_residual": g["tol_residual"]}
    path = os.path.join(ROOT, "tests", "golden", f"oracle_density_{cell.label}.npy")
    if rho is not None and os.path.exists(path):
        import numpy as np
        ref = np.load(path).astype(np.float64).reshape(-1)
        n = rho.double().cpu().numpy().reshape(-1)
        r["density_rel_l2"] = float(np.linalg.norm(n - ref) / np.linalg.norm(ref))
    return r


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import paper_2601_23002_gb300 as og
    from workloads import config_cell

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cell = config_cell(args.cell)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 126 MB L2

    def make(c, precision):
        plan = og.Plan(c.L, c.n, c.Z, c.T, rc=c.rc, precision=precision)
        dt = torch.float32 if precision == "fp32" else torch.float64
        rho = torch.empty(c.n ** 3, dtype=dt, device=dev)
        pos = torch.tensor(c.pos, dtype=torch.float64, device=dev)
        return plan, rho, pos

    def step(plan, rho, pos, shells=N_SHELLS):
        plan.structure_factor(pos)
        out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=TOL_F, tol_residual=TOL_R)
        if not out["converged"]:
            raise RuntimeError(f"snapshot did not converge: {out}")
        if shells:
            out["sei"] = plan.sei_shells(rho, shells)
        return out

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(plan, rho, pos, steps, shells=N_SHELLS):
        """Per-step device time from CUDA events on the library's stream; L2
        flushed before every step, outside the timed interval."""
        total_ms, evals, iters, last = 0.0, 0, 0, None
        for _ in range(steps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(plan, rho, pos, shells)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            evals += last["evaluations"]
            iters += last["iterations"]
        return total_ms, evals, iters, last

    def max_over_ranks(x):
        from paper_2601_23002_gb300.sharding import max_over_ranks as mor
        return mor(x, dev)

    res = {}
    plan, rho, pos = make(cell, "fp32")
    # FFT tile schedule from the library's autotuner (cached per grid size and
    # precision; outside the timed region, like the kernel table)
    plan.structure_factor(pos)
    if args.tiles:
        tiles = tuple(int(x) for x in args.tiles.split(","))
        plan.set_tiles(tiles)
    else:
        tiles = plan.autotune()[0]
    for _ in range(args.warmup):
        step(plan, rho, pos)
    # the timed region: launches are counted, but no event pair is recorded
    # around each launch (those pairs serialise the stream)
    plan.profile_enable(False)
    barrier()
    with ClockSampler(local) as clk:
        total_ms, evals, iters, last = timed(plan, rho, pos, args.steps)
    barrier()
    counts = plan.profile_read()
    total_ms_max = max_over_ranks(total_ms)
    # per-kernel device times for the roofline: the same steps again, with a
    # CUDA-event pair around every launch on the library's stream
    plan.profile_enable(True)
    barrier()
    prof_ms, _, _, _ = timed(plan, rho, pos, args.steps)
    barrier()
    prof = plan.profile_read()
    res["fp32"] = dict(total_ms=total_ms, total_ms_max=total_ms_max, evals=evals, iters=iters, last=last,
                       prof=prof, counts=counts, profiled_ms=prof_ms, clocks=clk.summary(), tiles=tiles,
                       error=error_vs_oracle(cell, last, rho))

    # end to end through the public API with host buffers: positions copied in
    # from pinned host memory; the converged density, the energies and S_ei
    # copied out, every step
    plan.profile_enable(False)
    host_pos_t = torch.empty(tuple(cell.pos.shape), dtype=torch.float64, pin_memory=True)
    host_pos_t.copy_(torch.from_numpy(np.ascontiguousarray(cell.pos, dtype=np.float64)))
    host_pos = host_pos_t.numpy()
    host_rho = torch.empty(cell.n ** 3, dtype=torch.float32, pin_memory=True)
    # Each step is timed on the host clock from the positions' copy-in to the
    # density on the host; the L2 flush between steps stays outside, as for value.
    barrier()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush_l2(flush)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        plan.structure_factor(host_pos)
        out = plan.minimize(rho, start_uniform=True, tol_F_per_ion=TOL_F, tol_residual=TOL_R)
        plan.sei_shells(rho, N_SHELLS)
        host_rho.copy_(rho, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_s += time.perf_counter() - t0
        if not out["converged"]:
            raise RuntimeError("e2e snapshot did not converge")
    e2e_s = max_over_ranks(e2e_s)
    res["e2e"] = dict(seconds=e2e_s, h2d=host_pos.nbytes,
                      d2h=host_rho.numel() * 4 + 11 * 8 + 2 * N_SHELLS * 8)
    plan.close()

    if not args.no_fp64:
        p64, r64, pos64 = make(cell, "fp64")
        _, ev64, it64, last64 = timed(p64, r64, pos64, 1)       # warm-up step (plan set-up paths)
        ms64, ev64, it64, last64 = timed(p64, r64, pos64, 1)
        res["fp64"] = dict(total_ms=max_over_ranks(ms64), evals=ev64, iters=it64, steps=1, last=last64,
                           error=error_vs_oracle(cell, last64, r64))
        p64.close()
        del r64
    if not args.no_cfg2:
        res["cfg2"] = run_cfg2(args, dev, make, timed, max_over_ranks)
    if not args.no_batched:
        res["batched"] = run_batched(args, dev)
    if args.serving > 0:
        res["serving"] = run_serving(args, dev)
    if not args.no_md:
        res["md"] = run_md(args, dev)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return cell, res


def run_cfg2(args, dev, make, timed, max_over_ranks):
    """The 64-H r_s = 2 theta = 1 cell on 128^3 (single snapshots, no S_ei):
    FP32 bulk and the plain FP64 path, each against the oracle's minimum."""
    from workloads import config_cell
    cell = config_cell(2)
    out = {"workload": "64 H ions (Z=1), r_s=2.0 bohr, theta=1.0, 128^3 grid, seeded random positions"}
    for precision, steps in (("fp32", max(3, args.steps)), ("fp64", 3)):
        if precision == "fp64" and args.no_fp64:
            continue
        plan, rho, pos = make(cell, precision)
        timed(plan, rho, pos, 2, 0)
        ms, ev, it, last = timed(plan, rho, pos, steps, 0)
        ms = max_over_ranks(ms)
        out[precision] = {"snapshots_per_s": steps / (ms * 1e-3), "evals_per_snapshot": ev / steps,
                          "evals_per_sec": ev / (ms * 1e-3), "ms_per_snapshot": ms / steps,
                          "error_vs_oracle": error_vs_oracle(cell, last, rho)}
        plan.close()
    return out


def run_batched(args, dev):
    """64 independent snapshots of uneven size (16-128 ions, Z in {1,3,4},
    r_s ~ U[1,3], theta ~ U[0.1,2], 48^3-96^3): the plain path (one after
    another on one stream) against the batched form (concurrent workers, one
    stream each).  Plans (kernel tables) are built and tiles tuned first,
    outside both timed regions."""
    import torch
    import paper_2601_23002_gb300 as og
    from paper_2601_23002_gb300.sharding import shard, snapshot_cost, max_over_ranks, sum_over_ranks
    from workloads import batch_cells
    # several GPUs: each rank takes its cost-balanced share of the snapshots;
    # throughput = all snapshots / the slowest rank's time
    rank, world, _ = dist_env()
    cells_all = batch_cells(args.batch_count)
    cells = [cells_all[i] for i in shard([snapshot_cost(c.n) for c in cells_all], world, rank)]
    plans = [og.plan_for_cell(c, precision="fp32") for c in cells]
    for p in plans:
        p.autotune()
    rhos = [torch.empty(c.n ** 3, dtype=torch.float32, device=dev) for c in cells]
    torch.cuda.synchronize(dev)
    og.minimize_batch(plans[:4], rhos[:4], concurrency=4)          # warm-up
    t0 = time.perf_counter()
    seq = [p.minimize(r, start_uniform=True, tol_F_per_ion=TOL_F, tol_residual=TOL_R) for p, r in zip(plans, rhos)]
    torch.cuda.synchronize(dev)
    t_seq = max_over_ranks(time.perf_counter() - t0, dev)
    out = {"workload": f"{len(cells_all)} snapshots, 16-128 ions, Z in {{1,3,4}}, r_s U[1,3], theta U[0.1,2], "
                       f"grids {sorted(set(c.n for c in cells_all))}",
           "ranks": world, "sequential_snapshots_per_s": len(cells_all) / t_seq}
    for conc in (8, 16, 32):
        t0 = time.perf_counter()
        res = og.minimize_batch(plans, rhos, concurrency=conc, tol_F_per_ion=TOL_F, tol_residual=TOL_R)
        torch.cuda.synchronize(dev)
        t = max_over_ranks(time.perf_counter() - t0, dev)
        out[f"batched_c{conc}_snapshots_per_s"] = len(cells_all) / t
        out[f"batched_c{conc}_converged"] = int(sum_over_ranks(sum(r["converged"] for r in res), dev))
    out["speedup_best"] = max(v for k, v in out.items() if k.startswith("batched_c") and k.endswith("per_s")) \
        / out["sequential_snapshots_per_s"]
    out["converged_sequential"] = int(sum_over_ranks(sum(r["converged"] for r in seq), dev))
    for p in plans:
        p.close()
    return out


# time per MD step the paper tabulates for its CPU runs (Methods, Table 2;
# 8 cores of 2x Xeon Gold 6240R): context, not a target of this machine
PAPER_MD_S_PER_STEP = {"md_H32_rs1": 0.08, "md_H14_rs2": 0.38, "md_H14_rs3.23": 2.39}


def run_md(args, dev, warm=10, steps=50):
    """Time per NVT MD step (electrons minimised from the previous density,
    forces, Nose-Hoover Verlet step) for the paper's three hydrogen MD cells:
    32 H at r_s = 1 (dt 0.02 fs), 14 H at r_s = 2 and 3.23 (dt 0.1 fs), theta = 1,
    T_ion = T, thermostat period 100 dt.  Wall time around ofdft_md_run (it
    synchronises), after `warm` equilibration steps."""
    import numpy as np
    import torch
    import paper_2601_23002_gb300 as og
    from workloads import hydrogen_md_cells, md_velocities, PROTON_MASS, SEED_BASE
    fs = 1.0 / 2.4188843265857e-2          # hbar/E_h per femtosecond
    out = {}
    for i, cell in enumerate(hydrogen_md_cells()):
        dt = (0.02 if cell.meta["rs"] == 1.0 else 0.1) * fs
        mass = np.full(cell.n_ion, PROTON_MASS)
        key = cell.label.rsplit("_n", 1)[0]
        row = {"n": cell.n, "n_ion": cell.n_ion, "T_eV": cell.T * 27.211386245988, "dt_fs": dt / fs,
               "paper_cpu_s_per_step": PAPER_MD_S_PER_STEP.get(key)}
        for precision in ("fp32", "fp64"):
            plan = og.plan_for_cell(cell, precision=precision)
            rho = torch.empty(cell.n ** 3, dtype=torch.float32 if precision == "fp32" else torch.float64,
                              device=dev)
            kw = dict(T_ion=cell.T, tau=100 * dt, tol_F_per_ion=TOL_F, tol_residual=TOL_R)
            vel = md_velocities(SEED_BASE + 7000 + i, mass, cell.T)
            a = plan.md_run(rho, cell.pos, vel, mass, warm, dt, start_uniform=True, **kw)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            b = plan.md_run(rho, a["pos"], a["vel"], mass, steps, dt, thermostat=a["thermostat"], **kw)
            t = time.perf_counter() - t0
            plan.close()
            row[precision] = {"ms_per_step": 1e3 * t / steps, "steps": steps,
                              "evals_per_step": float(np.mean(b["frames"]["evaluations"])),
                              "conserved_drift_per_ion": float(np.abs(b["frames"]["conserved"]
                                                                      - b["frames"]["conserved"][0]).max()
                                                               / cell.n_ion)}
        out[cell.label] = row
    return out


def run_serving(args, dev):
    """Poisson request stream (8-512 ions, 32^3-160^3): the plain sequential
    service rate on a sample of the stream first (every 10th request, at most
    200), then the continuous-batching server on the whole stream at 0.5, 0.9
    and 1.5 times that rate, and with every request waiting at the start
    (the server's capacity)."""
    import numpy as np
    from paper_2601_23002_gb300.serving import Server, run_sequential, summarize
    from workloads import serving_requests
    _, cells = serving_requests(args.serving)
    srv = Server(slots=16, precision="fp32")
    srv.prepare(cells)
    sample = cells[::10][:200]
    seq, t_seq = run_sequential(sample)
    mu = len(sample) / t_seq
    out = {"requests": len(cells), "sequential_snapshots_per_s": mu, "sequential_sample": len(sample),
           "sequential_converged": sum(1 for r in seq if r["converged"]), "slots": 16,
           "grids": sorted(set(c.n for c in cells))}
    for rho_f in (0.5, 0.9, 1.5):
        rng = np.random.default_rng(7)
        arrivals = np.cumsum(rng.exponential(1.0 / (rho_f * mu), size=len(cells)))
        done = srv.run(arrivals, cells)
        out[f"load_{rho_f}"] = summarize(done, srv.wall)
    # at a load of rho x the sequential rate the server can serve at most rho x
    # that rate; its capacity shows with every request waiting at the start
    done = srv.run(np.zeros(len(cells)), cells)
    out["load_saturated"] = summarize(done, srv.wall)
    out["served_over_sequential_at_1.5"] = out["load_1.5"]["snapshots_per_s"] / mu
    out["capacity_over_sequential"] = out["load_saturated"]["snapshots_per_s"] / mu
    return out


# ---------------------------------------------------------- roofline helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return float(e["dram_bytes_per_launch_full_size"])
    except Exception:
        pass
    return None


def roofline(prof):
    # dominant kernel = largest share of device time in the timed region
    name, (launches, ms, nbytes) = max(prof.items(), key=lambda kv: kv[1][1])
    peak, src = load_peaks()
    achieved = nbytes / launches / (ms / launches * 1e-3) / 1e9 if ms > 0 else 0.0
    total = sum(v[1] for v in prof.values())
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
            "traffic": load_traffic(name), "algorithmic_bytes_per_launch": nbytes / launches,
            "launches": launches, "avg_us": round(ms / launches * 1e3, 2), "share": round(ms / total, 4)}


# --------------------------------------------------------------- the oracle
_ORACLE_PLANS = {}


def oracle_sample(cell, n_evals: int, k_sf: int = 8, k_ew: int = 128):
    """The oracle's per-snapshot work, timed on a bounded sample: the ion
    structure factor (which V_loc is built from) on k_sf ions scaled by
    N_ion / k_sf (linear in the ions), the Ewald energy on k_ew ions scaled by
    (N_ion / k_ew)^2 (its pair sum), and n_evals FP64 functional evaluations
    at a perturbed density.  The evaluations run on a copy of the cell with
    k_sf ions of charge N_e / k_sf (the same N_e, nbar, T, L and grid: an
    evaluation's cost does not depend on the ions).  Returns seconds:
    (kernel-table set-up, per-snapshot set-up, per evaluation)."""
    import numpy as np
    from oracle.functional import Functional
    from oracle.cell import structure_factor, ewald_energy
    from workloads.cells import Cell
    ni = cell.n_ion
    k_sf, k_ew = min(k_sf, ni), min(k_ew, ni)
    key = (cell.label, k_sf)
    if key not in _ORACLE_PLANS:                   # the kernel table: built once, like a plan
        sub = Cell(L=cell.L, n=cell.n, Z=np.full(k_sf, cell.n_electrons / k_sf), pos=cell.pos[:k_sf],
                   theta=cell.theta, rc=cell.rc)
        t0 = time.perf_counter()
        _ORACLE_PLANS[key] = (Functional(sub), time.perf_counter() - t0)
    F, t_plan = _ORACLE_PLANS[key]
    t0 = time.perf_counter()
    structure_factor(cell.pos[:k_sf], cell.n, cell.L)
    t_sf = (time.perf_counter() - t0) * ni / k_sf
    t0 = time.perf_counter()
    ewald_energy(np.asarray(cell.Z[:k_ew], float), cell.pos[:k_ew], cell.L)
    t_ew = (time.perf_counter() - t0) * (ni / k_ew) ** 2
    rng = np.random.default_rng(0)
    psi = math.sqrt(F.nbar) * (1 + 0.05 * rng.standard_normal((cell.n,) * 3))
    t0 = time.perf_counter()
    for _ in range(n_evals):
        F.evaluate_psi(psi)
    t_eval = (time.perf_counter() - t0) / n_evals
    return t_plan, t_sf + t_ew, t_eval


def oracle_evals_per_snapshot(label: str):
    """(plain L-BFGS count, preconditioned count) of the oracle's converged
    minimum of this cell, from tests/golden/oracle_minima.json (None where
    absent)."""
    g = golden_minima()
    plain = g.get(label)
    pre = g.get(label + "_precond") or (plain if plain and plain.get("preconditioned") else None)
    if plain and plain.get("preconditioned"):
        plain = None
    return (int(plain["evaluations"]) if plain else None), (int(pre["evaluations"]) if pre else None)


def cpu_baseline(cell, fallback_evals: int, n_evals: int = 1):
    t_plan, t_snap, t_eval = oracle_sample(cell, n_evals)
    ev_plain, ev_pre = oracle_evals_per_snapshot(cell.label)
    ev = ev_plain or ev_pre or fallback_evals
    src = ("the plain oracle's own count" if ev_plain else
           "the preconditioned oracle's own count (a plain run takes hours)" if ev_pre else
           "the FP64 GPU run's count (no oracle count stored)")
    per_snap = t_snap + ev * t_eval
    out = {"value": 1.0 / per_snap, "unit": "snapshots/s", "cores": os.cpu_count(), "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": (f"oracle per-snapshot setup ({t_snap:.1f} s: structure factor on 8 ions x N_ion/8, "
                      f"Ewald on 128 ions x (N_ion/128)^2) + {n_evals} FP64 functional evaluation(s) of the "
                      f"{cell.n}^3 cell ({t_eval:.2f} s each), extrapolated with {ev} evaluations per converged "
                      f"snapshot ({src}, tests/golden/oracle_minima.json); kernel-table setup {t_plan:.1f} s "
                      f"excluded as on the GPU side")}
    if ev_plain and ev_pre:
        out["value_preconditioned"] = 1.0 / (t_snap + ev_pre * t_eval)
        out["evaluations_plain_preconditioned"] = [ev_plain, ev_pre]
    return out


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# -------------------------------------------------------------------- main
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        from workloads import config_cell
        cell = config_cell(args.cell)
        ev_plain, ev_pre = oracle_evals_per_snapshot(cell.label)
        ev = ev_plain or ev_pre or 100
        # each step: the bounded sample of oracle_sample (per-snapshot setup
        # on a sample of the ions + one FP64 evaluation), extrapolated to a
        # snapshot with the oracle's own evaluation count
        for _ in range(args.warmup):
            oracle_sample(cell, 1)
        per = []
        for _ in range(args.steps):
            _, t_snap, t_eval = oracle_sample(cell, 1)
            per.append(t_snap + ev * t_eval)
        value = len(per) / sum(per)
        sample = (f"per step: oracle per-snapshot setup (structure factor on 8 ions x N_ion/8, Ewald on 128 "
                  f"ions x (N_ion/128)^2) + 1 FP64 evaluation of the {cell.n}^3 cell, extrapolated with {ev} "
                  f"evaluations per snapshot (the {'plain' if ev_plain else 'preconditioned'} oracle's own count)")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "snapshots/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per) / len(per),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config_dict(world, world * args.steps, cell),
                "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "cpu_model": cpu_model(),
                                 "value": value, "sample": sample},
                "e2e": {"value": value, "unit": "snapshots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    cell, res = run_ours(args, rank, world, local)
    if rank != 0:
        return 0
    r32 = res["fp32"]
    N = cell.n ** 3
    secs = r32["total_ms_max"] * 1e-3
    snaps = world * args.steps
    value = snaps / secs
    evals_per_s = world * r32["evals"] / secs
    b_eval = 14 * N * 4
    prof = r32["prof"]
    launches = sum(v[0] for v in r32["counts"].values())
    line = {
        "metric": METRIC, "value": value, "unit": "snapshots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["total_ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 sums and line search)", "data": "synthetic",
        "config": config_dict(world, snaps, cell),
        "evals_per_sec": evals_per_s, "evals_per_snapshot": r32["evals"] / args.steps,
        "iterations_per_snapshot": r32["iters"] / args.steps,
        "fft_tiles": {"z_rows": r32["tiles"][0], "y_cols": r32["tiles"][1], "x_cols": r32["tiles"][2],
                      "source": "--tiles" if args.tiles else "ofdft_autotune"},
        "effective_hbm_gbs": evals_per_s / world * b_eval / 1e9,
        "effective_hbm_note": "14 N w bytes per evaluation (w = 4) x evals/s, per GPU",
        "final_energy": {k: r32["last"][k] for k in ("F_total", "residual", "N_e")},
        "error_vs_oracle": r32["error"],
        "clocks": r32["clocks"],
        "e2e": {"value": snaps / res["e2e"]["seconds"], "unit": "snapshots/s",
                "h2d_bytes_per_step": res["e2e"]["h2d"], "d2h_bytes_per_step": res["e2e"]["d2h"]},
        "gpu_launches": launches,
        "roofline": roofline(prof),
        "profiled_ms_per_step": r32["profiled_ms"] / args.steps,
        "profiled_note": "kernels and roofline come from a second pass over the same steps with an event pair around every launch; value and ms_per_step from the pass without them",
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 3), "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] else None}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
    }
    if "fp64" in res:
        r = res["fp64"]
        line["fp64"] = {"value": world * r["steps"] / (r["total_ms"] * 1e-3), "unit": "snapshots/s",
                        "evals_per_sec": world * r["evals"] / (r["total_ms"] * 1e-3),
                        "evals_per_snapshot": r["evals"] / r["steps"], "steps": r["steps"],
                        "F_total": r["last"]["F_total"], "error_vs_oracle": r["error"],
                        "fp32_minus_fp64_F_per_ion": (r32["last"]["F_total"] - r["last"]["F_total"]) / cell.n_ion}
    if "cfg2" in res:
        line["cfg2"] = res["cfg2"]
    if "batched" in res:
        line["batched"] = res["batched"]
    if "serving" in res:
        line["serving"] = res["serving"]
    if "md" in res:
        line["md"] = res["md"]
    if world == 1 and not args.no_cpu_baseline:
        fallback = int(line.get("fp64", {}).get("evals_per_snapshot", r32["evals"] / args.steps))
        line["cpu_baseline"] = cpu_baseline(cell, fallback)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())

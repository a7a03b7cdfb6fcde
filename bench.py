#!/usr/bin/env python
"""Throughput of the EM-PIC hot path on GB300.

Default workload: 3D3V periodic thermal plasma, 512x256x256 cells, 8 particles
per cell (268,435,456 electrons), u_th = 0.05 c, dx = 0.1 c/w_p, dt = 0.99 of the
Courant limit, in the FP32 cell-offset tiled form.  One "step" is one full PIC
step: gather + Boris push + move + charge-conserving deposit (with the per-tile
binning), current fold, field solve.  Particles and fields are resident in HBM
(the particle store alone is ~9 GB, far larger than L2).

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Prints one JSON line (rank 0).  With N > 1 (launched by torchrun) every rank runs
an independent replica with its own seed ("replicas only": the workload does
not exchange data between GPUs); the timed region is bracketed by barriers and
the max over ranks is reported.
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

METRIC = "particle pushes/s (gather+push+deposit) and % HBM roofline, FP32 vs FP64 at stated error"
UNIT = "particle-pushes/s"
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes per particle-step: particle record read + written, plus the
# per-cell field reads (6 E/B components) and current read-modify-write (3)
# amortised over the particles of a cell
REC_BYTES = {("fp32", 3): 28, ("fp32", 2): 24, ("fp64", 3): 48, ("fp64", 2): 40}


def alg_bytes_per_particle(prec: str, ndim: int, ppc: int) -> float:
    w = 4 if prec == "fp32" else 8
    return 2 * REC_BYTES[(prec, ndim)] + (6 * w + 3 * w * 2) / ppc


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ppc", type=int, default=8, choices=[1, 2, 4, 8, 16])
    p.add_argument("--nx", default="512,256,256")
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--tile", default="auto", help="tile shape in cells, e.g. 4,4,4 (auto: the library's choice)")
    p.add_argument("--smooth", type=int, default=0, help="(1,2,1) passes per direction")
    p.add_argument("--sort-period", type=int, default=0,
                   help="steps per cell re-sort of the tiles (0: the library's default)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--scan-steps", type=int, default=500,
                   help="timed steps of the batched-scan comparison (64 wakefield runs, batched vs one by one; "
                        "the scan's own length is 500)")
    p.add_argument("--no-scan", action="store_true")
    p.add_argument("--wake-steps", type=int, default=200,
                   help="timed steps of the 2D laser-wakefield workload (moving window)")
    p.add_argument("--no-wake", action="store_true")
    p.add_argument("--cyl-steps", type=int, default=20,
                   help="timed steps of the r-z (2D cylindrically symmetric) plasma column, FP64")
    p.add_argument("--no-cyl", action="store_true")
    return p.parse_args()


# ---------------------------------------------------------------- environment
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if "Active" in f[5 + k] and "Not" not in f[5 + k]:
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_tiled.cu", "tile_dev.cuh", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_1503_00276_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n_particles: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel]
        if rec.get("source_hash") != source_hash():
            return None
        return rec["dram_bytes_per_particle"] * n_particles
    except Exception:
        return None


# ---------------------------------------------------------------- workloads
def make_workload(args, rank: int):
    import workload
    nx = tuple(int(v) for v in args.nx.split(","))
    g, sps, steps = workload.config3(args.ppc, seed=20004 + rank, nx=nx)
    g.smooth_level = (args.smooth,) * 3
    return g, sps, steps


def describe(args, n_p: int, info=None, arm: str = "ours"):
    """The workload of the line.  info: the simulation's pic_info (tile shape
    and sort period as in use); arm "reference": the FP64 CPU oracle."""
    nx = [int(v) for v in args.nx.split(",")]
    if arm == "reference":
        form, prec = "FP64 CPU oracle (reference arm)", "fp64 (oracle)"
    else:
        form, prec = ("FP32 cell-offset tiled" if args.precision == "fp32" else "FP64 plain"), args.precision
    tile = None
    if arm != "reference" and args.precision == "fp32":
        tile = list(info["tile"]) if info else args.tile
    return {
        "workload": (f"3D3V periodic thermal plasma {nx[0]}x{nx[1]}x{nx[2]} cells, {args.ppc} ppc "
                     f"({n_p:,} electrons), u_th=0.05c, dx=0.1 c/w_p, dt=0.99 Courant, {form}"),
        "grid": nx, "ppc": args.ppc, "precision": prec,
        "tile": tile,
        "smoothing_passes": args.smooth,
        "sort_period": (int(info["sort_period"]) if info else (args.sort_period or 1)) if arm != "reference" else None,
        "l2": "inputs larger than L2 (particle store >= 7.5 GB vs 129 MB L2)",
        "steps_in_config": 200,
    }


# ---------------------------------------------------------------- replicas
def rank_reducers(dist, device):
    """(max over ranks, sum over ranks) of a host float, through an all-reduce
    of a one-element FP64 tensor on ``device``; identities without a process
    group.  Each rank runs its own replica (no data-path collective): the job's
    time is the slowest rank's and its units are the sum over the ranks."""
    import torch

    def reduce(v: float, op) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    if dist is None:
        return (lambda v: v), (lambda v: v)
    return (lambda v: reduce(v, dist.ReduceOp.MAX)), (lambda v: reduce(v, dist.ReduceOp.SUM))


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1503_00276_gb300 as pg
    import workload

    g, sps, _ = make_workload(args, rank)
    n_p = workload.n_particles(g, sps[0])
    tile = None if args.tile == "auto" else tuple(int(v) for v in args.tile.split(","))
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    max_over_ranks, sum_over_ranks = rank_reducers(dist, "cuda")

    def timed(sim, steps, warmup, clocks=None):
        for _ in range(warmup):
            sim.step(1)
        sim.timing_enable(True)
        sim.timing_read(reset=True)
        barrier()
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sim.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        tim = sim.timing_read(reset=True)
        sim.timing_enable(False)
        return ms, tim, clk

    peak, peak_kind = measured_peak()
    prec = args.precision
    sim = pg.Simulation(g, sps, precision=prec, tile=tile if prec == "fp32" else None,
                        sort_period=args.sort_period)
    clocks = ClockSampler(local)
    ms, tim, clk = timed(sim, args.steps, args.warmup, clocks)
    diag = sim.diag()
    info = sim.info()
    sim.close()
    del sim
    ms_max = max_over_ranks(ms)
    total_units = sum_over_ranks(n_p * args.steps)
    value = total_units / (ms_max / 1e3)
    k1_ms, k1_n = tim["particles"]
    k1_avg_s = k1_ms / max(k1_n, 1) / 1e3
    bpp = alg_bytes_per_particle(prec, 3, args.ppc)
    achieved = n_p * bpp / k1_avg_s / 1e9
    kname = "k_tile_push" if prec == "fp32" else "k_plain_push"
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": profiled_traffic(kname, n_p),
            "kernel": kname, "algorithmic_bytes_per_particle": bpp, "peak_source": f"{peak_kind} hbm_gbs",
            "k1_ms_per_launch": round(k1_avg_s * 1e3, 4), "step_roofline_frac": round(
                n_p * bpp / (ms / args.steps / 1e3) / 1e9 / peak, 4)}
    launches = int(tim["launches"][1])

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
           "data": "synthetic (seeded lattice + Maxwellian loader, no dataset)", "config": describe(args, n_p, info),
           "roofline": roof, "clocks": clk, "gpu_launches": launches,
           "stages_ms_per_step": {k: round(v[0] / max(args.steps, 1), 4) for k, v in tim.items()
                                  if k not in ("launches",)},
           "diag_after": {"gauss_resid_max": diag["gauss_resid_max"],
                          "rho_particles_abs_max": diag["rho_particles_abs_max"],
                          "error_flags": diag["error_flags"]}}

    # FP64 plain form on the same GPU (speed-up statement)
    if not args.no_fp64 and prec == "fp32":
        s64 = pg.Simulation(g, sps, precision="fp64")
        ms64, tim64, _ = timed(s64, args.fp64_steps, 1)
        s64.close()
        del s64
        ms64 = max_over_ranks(ms64)
        v64 = sum_over_ranks(n_p * args.fp64_steps) / (ms64 / 1e3)
        k64 = tim64["particles"][0] / max(tim64["particles"][1], 1) / 1e3
        b64 = alg_bytes_per_particle("fp64", 3, args.ppc)
        out["fp64_plain"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps,
                             "steps": args.fp64_steps,
                             "roofline_frac": round(n_p * b64 / k64 / 1e9 / peak, 4),
                             "k1_ms_per_launch": round(k64 * 1e3, 3),
                             "fp32_speedup": value / v64}

    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, g, sps, n_p, tile, barrier, max_over_ranks, sum_over_ranks)

    if not args.no_scan:
        out["batch_scan"] = run_batch_scan(args, max_over_ranks)
    if not args.no_wake:
        out["wakefield_2d"] = run_wakefield(args, max_over_ranks)
        out["beam_wake_3d"] = run_beam_wake(args, max_over_ranks)
    if not args.no_cyl:
        out["cylindrical_2d"] = run_cylindrical(args, max_over_ranks)

    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = run_cpu_baseline(args, budget_s=15.0)
    # the side measurements in one flat object at the end of the line
    summ = {"kernel_ms": roof["k1_ms_per_launch"], "hbm_frac": roof["frac"]}
    if "fp64_plain" in out:
        summ["fp64_plain_pushes_per_s"] = out["fp64_plain"]["value"]
        summ["fp32_over_fp64_plain"] = round(out["fp64_plain"]["fp32_speedup"], 2)
    if "batch_scan" in out:
        summ["batch_pushes_per_s"] = out["batch_scan"]["batched"]["value"]
        summ["batch_over_one_by_one"] = round(out["batch_scan"]["speedup"], 3)
    for k in ("wakefield_2d", "beam_wake_3d", "cylindrical_2d"):
        if k in out:
            summ[k + "_pushes_per_s"] = out[k]["value"]
    if "cylindrical_2d" in out:
        summ["rz_fp32_over_fp64"] = round(out["cylindrical_2d"]["fp32_speedup"], 2)
        summ["rz_gauss_change_over_rho"] = out["cylindrical_2d"]["fp32"]["gauss_resid_change_over_rho_max"]
    if "cpu_baseline" in out:
        summ["oracle_pushes_per_s"] = out["cpu_baseline"]["value"]
        summ["oracle_cores"] = out["cpu_baseline"]["cores"]
    out["summary"] = summ
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_cylindrical(args, max_over_ranks):
    """The r-z (2D cylindrically symmetric) mode: a thermal plasma column of
    2048 x 512 cells of 0.1 c/w_p out to a conducting wall, 4 rings per cell
    (4.2M), u_th = 0.05, fixed ion background; the FP32 tiled form (the
    line's value) and the FP64 plain form."""
    import torch

    import paper_1503_00276_gb300 as pg
    import workload

    g, sps, _ = workload.config_cyl()
    K, W = args.cyl_steps, 3
    stream = torch.cuda.current_stream()
    res = {}
    for prec in ("fp32", "fp64"):
        sim = pg.Simulation(g, sps, precision=prec)
        # the column starts with E = 0: the first node row off the axis carries
        # a residual of 0.375 (the fold of the mirror row); it must not change
        d0 = sim.diag()
        sim.timing_enable(True)
        sim.step(W)
        torch.cuda.synchronize()
        sim.timing_read(reset=True)
        n0 = sim.n_particles()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        tim = sim.timing_read()
        d = sim.diag()
        info = sim.info()
        sim.close()
        res[prec] = {"value": n0 * K / (ms / 1e3), "ms_per_step": ms / K, "tile": list(info["tile"]),
                     "stages_ms_per_step": {k: round(v[0] / K, 4) for k, v in tim.items() if k != "launches"},
                     "gauss_resid_max_before": d0["gauss_resid_max"], "gauss_resid_max_after": d["gauss_resid_max"],
                     "gauss_resid_change_over_rho_max": abs(d["gauss_resid_max"] - d0["gauss_resid_max"]) /
                     d["rho_particles_abs_max"], "rho_abs_max_after": d["rho_abs_max"]}
    out = {"workload": f"r-z plasma column 2048x512 cells, dz = dr = 0.1, 2x2 rings per cell ({n0:,}), "
                       "u_th=0.05, conducting wall", "steps": K, "warmup": W, "unit": UNIT,
           "value": res["fp32"]["value"], "precision": "fp32 tiled (value); fp64 plain beside it"}
    out.update({"fp32": res["fp32"], "fp64": res["fp64"], "fp32_speedup": res["fp32"]["value"] / res["fp64"]["value"]})
    return out


def run_wakefield(args, max_over_ranks):
    """The 2D laser-wakefield workload in the FP32 form: 2048 x 256 cells,
    4.2M electrons, laser a0 = 2, window moving at c (a one-cell shift with
    a fresh front column about every 1.5 steps)."""
    import torch

    import paper_1503_00276_gb300 as pg
    import workload

    g, sps, las, _ = workload.config1()
    sim = pg.Simulation(g, sps, precision="fp32")
    sim.add_laser(las)
    K, W = args.wake_steps, 5
    stream = torch.cuda.current_stream()
    sim.timing_enable(True)
    sim.step(W)
    torch.cuda.synchronize()
    sim.timing_read(reset=True)
    n0 = sim.n_particles()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1))
    tim = sim.timing_read()
    d = sim.diag()
    info = sim.info()
    sim.close()
    return {"workload": "2D3V laser wakefield 2048x256 cells, dx 0.05 x 0.2, 8 ppc cold electrons "
                        f"({n0:,}), a0=2, omega0=10, spot 4, window moving at c", "steps": K, "warmup": W,
            "value": n0 * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K, "tile": list(info["tile"]),
            "stages_ms_per_step": {k: round(v[0] / K, 4) for k, v in tim.items() if k != "launches"},
            "rebuilds": int(tim["rebuild"][1]),
            "field_energy_after": d["field_energy"], "n_particles_after": d["n_particles"]}


def run_beam_wake(args, max_over_ranks):
    """The 3D beam-driven wake in the FP32 form: 256 x 128 x 128 cells, 33.5M
    plasma electrons plus a 4.2M-macroparticle bi-Gaussian driver at
    gamma = 60000, window moving at c."""
    import torch

    import paper_1503_00276_gb300 as pg
    import workload

    g, sps, (bx, bu, bq), _ = workload.config2()
    sim = pg.Simulation(g, sps, precision="fp32", explicit=[None, (bx, bu, bq)])
    K, W = max(args.wake_steps // 4, 10), 5
    stream = torch.cuda.current_stream()
    sim.timing_enable(True)
    sim.step(W)
    torch.cuda.synchronize()
    sim.timing_read(reset=True)
    n0 = sim.n_particles(0) + sim.n_particles(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1))
    tim = sim.timing_read()
    info = sim.info()
    sim.close()
    return {"workload": "3D3V beam-driven wake 256x128x128 cells, dx 0.05 x 0.1 x 0.1, 8 ppc cold plasma + "
                        f"bi-Gaussian driver gamma=60000, sigma 1 x 0.3, n_b/n_0=5 ({n0:,} particles), window "
                        "moving at c", "steps": K, "warmup": W, "value": n0 * K / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / K, "tile": list(info["tile"]),
            "stages_ms_per_step": {k: round(v[0] / K, 4) for k, v in tim.items() if k != "launches"},
            "rebuilds": int(tim["rebuild"][1])}


def run_batch_scan(args, max_over_ranks):
    """The batched parameter scan: 64 independent 2D3V wakefield runs of uneven
    size (81.7M electrons in all; windows moving at c, in-box pulses of a0 0.5-3
    at omega0 = 10 w_p), advanced as one batch (one CUDA graph per step: one
    tile-kernel launch for every member's particles and one launch per field
    stage for all members) versus one by one through pic_step.  Both read the
    device status back after every step.  Each arm takes 3 untimed steps, then
    --scan-steps timed ones."""
    import torch

    import paper_1503_00276_gb300 as pg
    import workload

    sims, c4_steps = workload.config4()
    n_p = sum(workload.n_particles(g, s[0]) for g, s, _ in sims)
    K, W = args.scan_steps, 3
    stream = torch.cuda.current_stream()
    # tile shape and blocks per SM by the library's autotuner (each candidate
    # is the whole batch without its pulses, 2 + 3 steps)
    best, tried = pg.batch_autotune(sims, warmup=2, steps=3)

    def timed(step):
        step(W)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    batch = pg.Batch(sims, tile=best["tile"], ctas_per_sm=best["ctas_per_sm"])  # pulses added per member
    ms_b = max_over_ranks(timed(batch.step))
    info = batch.info()
    n_end = sum(batch.sim(i).n_particles() for i in range(len(sims)))
    batch.close()
    del batch
    ms_s = 0.0
    for g, sps, las in sims:
        s = pg.Simulation(g, sps, precision="fp32", tile=best["tile"], ctas_per_sm=best["ctas_per_sm"])
        s.add_laser(las)
        ms_s += timed(s.step)
        s.close()
    ms_s = max_over_ranks(ms_s)
    return {"workload": "64 x 2D3V wakefield runs drawn from the scan seed (128x64 .. 1024x512 cells, 4-32 ppc, "
                        "density 0.5-2, laser a0 0.5-3 at omega0 = 10 w_p, windows moving at c), 81.7M electrons",
            "members": len(sims), "particles": n_p, "particles_at_end": n_end, "steps": K, "warmup": W,
            "config_steps": c4_steps, "tile": list(info["tile"]),
            "autotune": {"chosen": best, "tried": tried},
            "batched": {"value": n_p * K / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b / K,
                        "launches_per_step": info["launches"] / max(info["steps"], 1)},
            "sequential": {"value": n_p * K / (ms_s / 1e3), "unit": UNIT, "ms_per_step": ms_s / K},
            "speedup": ms_s / ms_b}


def run_e2e(args, g, sps, n_p, tile, barrier, max_over_ranks, sum_over_ranks):
    """One job through the public API: upload the initial particles from pinned
    host memory (pic_init with explicit arrays), advance K steps reading the FP64
    diagnostics back every step, copy all particles back to pinned host memory."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import paper_1503_00276_gb300 as pg
    import workload

    x = torch.empty((n_p, 3), dtype=torch.float64, pin_memory=True)
    u = torch.empty((n_p, 3), dtype=torch.float64, pin_memory=True)
    xn, un = x.numpy(), u.numpy()
    chunk = 1 << 22

    def gen(first):
        idx = np.arange(first, min(first + chunk, n_p), dtype=np.int64)
        a, b = workload.load_particles(g, sps[0], idx)
        xn[first:first + idx.size] = a
        un[first:first + idx.size] = b

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        list(ex.map(gen, range(0, n_p, chunk)))
    q = workload.macro_charge(g, sps[0])
    steps = args.steps
    barrier()
    t0 = time.perf_counter()
    sim = pg.Simulation(g, sps, precision=args.precision, explicit=[(xn, un, q)],
                        tile=tile if args.precision == "fp32" else None, sort_period=args.sort_period)
    ta = time.perf_counter()
    t_diag = 0.0
    for _ in range(steps):
        sim.step(1)
        td = time.perf_counter()
        sim.diag()
        t_diag += time.perf_counter() - td
    tb = time.perf_counter()
    got = sim.particles_into(xn, un)
    sim.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    barrier()
    assert got == n_p
    sec = max_over_ranks(t1 - t0)
    value = sum_over_ranks(n_p * steps) / sec
    h2d = 2 * n_p * 3 * 8
    d2h = 2 * n_p * 3 * 8 + steps * 80
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "job": f"pic_init from pinned host FP64 arrays + {steps} x (pic_step + pic_diag) + pic_particles to "
                   f"pinned host", "seconds": sec,
            "phases_s": {"init_upload": round(ta - t0, 3), "steps": round(tb - ta - t_diag, 3),
                         "diag": round(t_diag, 3), "readback_free": round(t1 - tb, 3)}}


# ---------------------------------------------------------------- oracle arms
def oracle_sample(cells_target: int, ppc: int, seed: int = 20004):
    """A periodic sub-box of the workload (same dx, u_th, ppc) with about
    cells_target cells."""
    import workload
    dims = [8, 8, 8]
    k = 0
    while dims[0] * dims[1] * dims[2] * 2 <= cells_target and max(dims) < 512:
        dims[k % 3] *= 2
        k += 1
    dims.sort(reverse=True)
    g, sps, _ = workload.config3(ppc, seed=seed, nx=tuple(dims))
    return g, sps, dims


def _oracle_process(cells, ppc, seed, warmup, steps, barrier, queue):
    """One host process of the all-core oracle run: its own periodic sub-box
    (own seed), warm-up steps, then (after every process is ready) timed
    steps; reports (particles, steps, start, end) in wall-clock time."""
    sys.path.insert(0, ROOT)
    import oracle
    import workload
    g, sps, dims = oracle_sample(cells, ppc, seed)
    st = oracle.from_workload(g, sps)
    n = workload.n_particles(g, sps[0])
    st.step(max(warmup, 1))
    barrier.wait()
    t0 = time.time()
    st.step(steps)
    queue.put((n, steps, t0, time.time(), dims))


def oracle_all_cores(cells, ppc, warmup, steps, nproc):
    """The unchanged oracle on nproc host cores at once: independent processes
    (started with spawn; no state shared with this GPU process) on disjoint
    periodic sub-boxes.  Returns (pushes/s over the common timed span,
    particles per process, box dims)."""
    import multiprocessing as mp
    import oracle
    oracle.build()  # the processes load the built library
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(nproc)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_process, args=(cells, ppc, 20004 + 17 * k, warmup, steps, barrier, queue))
             for k in range(nproc)]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    total = sum(n * k for n, k, _, _, _ in res)
    span = max(e for _, _, _, e, _ in res) - min(b for _, _, b, _, _ in res)
    return total / span, res[0][0], res[0][4], span


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_cpu_baseline(args, budget_s: float):
    """The FP64 oracle on the host: one thread on a 64x64x32 sub-box (about
    budget_s), then every host core at once (the core count read here), each
    on its own 32x32x32 sub-box for about budget_s."""
    import oracle
    import workload
    g, sps, dims = oracle_sample(1 << 17, args.ppc)
    st = oracle.from_workload(g, sps)
    n = workload.n_particles(g, sps[0])
    t0 = time.perf_counter()
    st.step(1)
    one = time.perf_counter() - t0
    more = max(0, int(budget_s / max(one, 1e-3)) - 1)
    t1 = time.perf_counter()
    if more:
        st.step(more)
    total = (time.perf_counter() - t1) + one
    steps = more + 1
    single = {"value": n * steps / total, "cores": 1,
              "sample": f"{dims[0]}x{dims[1]}x{dims[2]} periodic sub-box, {n:,} electrons, {steps} steps, "
                        f"{total:.1f} s"}
    cores = host_cores()
    # each process: a quarter of the single-thread box, steps for ~budget_s
    per_step = one / 4.0
    msteps = max(2, int(budget_s / max(per_step, 1e-3)))
    val, np_, mdims, span = oracle_all_cores(1 << 15, args.ppc, 1, msteps, cores)
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} host processes at once, each a {mdims[0]}x{mdims[1]}x{mdims[2]} periodic sub-box of "
                      f"the workload at {args.ppc} ppc ({np_:,} electrons), {msteps} full FP64 steps, {span:.1f} s",
            "single_thread": single}


def run_reference(args):
    """The reference arm: the FP64 oracle on every host core (independent
    processes on disjoint periodic sub-boxes of the workload); each of the
    K + W steps advances every sub-box one step, sized so that the run takes
    about 150 s."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import workload
    k, w = args.steps, args.warmup
    cores = host_cores()
    # ~1.2 us per particle-step of the oracle on one core
    cells = int(150.0 / max(k + w, 1) / (args.ppc * 1.2e-6))
    cells = max(512, min(cells, 1 << 21))
    g_full, sp_full, _ = make_workload(args, 0)
    value, n, dims, span = oracle_all_cores(cells, args.ppc, w, k, cores)
    sample = (f"{cores} host processes at once, each a {dims[0]}x{dims[1]}x{dims[2]} periodic sub-box of the workload, "
              f"{args.ppc} ppc ({n:,} electrons) per process, FP64 oracle, {w} warm-up + {k} timed steps")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": k,
           "warmup": w, "ms_per_step": span / max(k, 1) * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded lattice + Maxwellian loader)",
           "config": describe(args, workload.n_particles(g_full, sp_full[0]), arm="reference"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

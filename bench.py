#!/usr/bin/env python3
"""Benchmark of the avalanche-overlay hot path on GB300.

One step = the whole workflow over the 8192 x 8192 synthetic DEM (fBm plus a
carved valley network, 10 m cells, uint16 decimetres): decode -> normals ->
release (about 5% of the cells) -> 256 particles per release cell (step cap
8000) -> velocity -> 6-level mipmap, with the DEM already resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl awo|reference]

Prints one JSON line (rank 0).  ``value`` is trajectory steps (recorded
particle moves) per second over the whole step; ``ms_per_step`` is ms per
overlay.  ``--impl reference`` times the CPU oracle on the host cores on
bounded samples of the same workload.  Under torchrun every rank runs its own
replica of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trajectory-steps/s and ms/overlay at 8192^2 DEM on 1 GB300; % of gather roofline"
UNIT = "trajectory-steps/s"

# Bytes per visit of the particle kernel that the roofline counts as
# algorithmic: a 2x2 FP32 height footprint (16 B) plus two 4-byte reductions
# (count, energy) for a move, or one reduction plus the 4-byte release-index
# read for a release visit.
ALG_BYTES_PER_VISIT = 24

# Algorithmic lane operations per visit of the particle kernel, counted from
# the formulas of the move: half a Philox4x32-10 block (a block -- 10 rounds
# x (2 multiply high + 2 multiply low + 4 xor + 2 key add) = 100 -- yields
# the four words of two moves) = 50, and the move's two uniforms 8; bilinear
# height 11; gradient and its normalisation 17; direction 17; move and
# domain test 8; energy and stop test 6; visited cell 5; floors 4.
ALG_OPS_PER_VISIT = 126

# Counters of the particle kernel from one ncu capture of a 6144^2 crop launch
# of the 8192^2 workload (bench.py --workload large --crop 6144), per visit
# (release visit or move attempt) of that launch, keyed by the SHA-256 prefix
# of the kernel's code (comments removed) they were taken on; a changed kernel
# reports them as null until it is captured again:
#   dram: dram__bytes_read.sum + dram__bytes_write.sum
#   lts_frac: lts__throughput.avg.pct_of_peak_sustained_elapsed / 100, the L2's
#     own utilisation against its peak -- the L2 gather/reduction roofline
#     fraction of the kernel
#   red_sectors, read_sectors: lts__t_sectors_srcunit_tex_op_red.sum and
#     lts__t_sectors_srcunit_tex_op_read.sum (the visits' reductions, and the
#     footprint reads that miss in the L1/texture cache, as the SMs send them)
#   atomic_busy: lts__d_atomic_input_cycles_active.avg.pct_of_peak_sustained_elapsed
#     / 100, the share of cycles the L2's reduction units take input
KERNEL_COUNTERS: dict[str, dict[str, float]] = {
    "21bee4ee6bfef80c": {"dram": (917.063680e6 + 189.185280e6) / 1754008332, "lts_frac": 0.77099731,
                         "red_sectors": 2177706165 / 1754008332, "read_sectors": 32575163 / 1754008332,
                         "atomic_busy": 0.52413501},
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["awo", "reference"], default="awo")
    ap.add_argument("--workload", choices=["large", "mid", "tiny", "batched", "served", "diff", "parabola",
                                           "stages"], default="large")
    ap.add_argument("--batch-n", type=int, default=64, help="regions of the batched/served workload")
    ap.add_argument("--rate", type=float, default=200.0, help="Poisson arrival rate of the served workload (1/s)")
    ap.add_argument("--crop", type=int, default=0, help="use the top-left N x N crop of the workload's DEM")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-instances", type=int, default=3, help="workflow instances of the pipelined end-to-end run")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the batched, served, differentiable and parabola runs of the default line")
    ap.add_argument("--cpu-threads", type=int, default=0, help="host threads of the oracle (0 = all cores)")
    ap.add_argument("--release-log2", type=int, default=0,
                    help="evaluate release points on a texture at 2^r x the DEM resolution (large/mid/tiny)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# ranks
# ----------------------------------------------------------------------------
class Ranks:
    def __init__(self):
        import torch
        import torch.distributed as dist

        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = dist if self.world > 1 else None
        self.torch = torch
        backend = None
        if self.dist is not None:
            backend = os.environ.get("AWO_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
        on_gpu = torch.cuda.is_available() and (self.dist is None or backend == "nccl")
        self.device = torch.device("cuda", self.local) if on_gpu else torch.device("cpu")

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def reduce(self, x: float, op: str) -> float:
        if self.dist is None:
            return x
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == "max" else self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
_REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
                0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.sel = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            if uuid:
                self.sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            self.sel = []

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="awo_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", *self.sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             int(parts[4], 16) if parts[4].startswith("0x") else 0, parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[2] > 0 and not (r[3] & 0x1)] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in loaded:
            for bit, name in _REASON_BITS.items():
                if r[3] & bit and name != "gpu_idle":
                    reasons.add(name)
            for name, flag in zip(names, r[4]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(loaded), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def _workload(name: str, crop: int = 0):
    from paper_2506_23364_gb300 import inputs
    w = {"large": inputs.large, "mid": inputs.mid, "tiny": inputs.tiny}[name]()
    return inputs.crop(w, crop) if crop else w


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _kernel_sha() -> str:
    """Hash of the particle kernel's sources (the kernel and its per-move
    code), comments and blank space removed, so that only code changes
    invalidate counters taken on an earlier build."""
    h = hashlib.sha256()
    for name in ("awo_simulate.cu", "awo_particle.cuh"):
        with open(os.path.join(ROOT, "paper_2506_23364_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _probe_peaks(torch, awo) -> dict:
    """L2 scattered-load and scattered-reduction rates, best of 5 (events)."""
    buf = torch.zeros(8 << 20, dtype=torch.int32, device="cuda")  # 32 MiB: L2-resident
    sink = torch.empty(awo.awo_probe_threads(), dtype=torch.int32, device="cuda")
    iters = 256
    out = {}
    for name, fn, per in (("l2_gather", lambda: awo.awo_probe_l2_gather(buf, iters, sink), 4),
                          ("l2_red", lambda: awo.awo_probe_l2_red(buf, iters), 2)):
        fn()
        torch.cuda.synchronize()
        best = math.inf
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        out[name + "_per_s"] = awo.awo_probe_threads() * iters * per / best
    return out


def _oracle_rate(oracle, h, cs, cells, p, threads, rng) -> float:
    """Release cells per second of the threaded oracle, from samples grown
    until one takes at least a second."""
    import numpy as np

    k = min(cells.size, 64 * threads)
    while True:
        probe = np.sort(rng.choice(cells, k, replace=False))
        t0 = time.perf_counter()
        oracle.simulate_threaded(h, cs, probe, p, threads=threads, merge=False)
        dt = time.perf_counter() - t0
        if dt >= 1.0 or k >= cells.size:
            return k / max(dt, 1e-6)
        k = min(cells.size, int(k * max(2.0, 1.5 / max(dt, 1e-3))))


def _cpu_baseline(w, seconds: float, threads: int | None = None) -> dict:
    """The oracle, as it stands, on the host cores over a random sample of the
    workload's release cells (all particles of each sampled cell)."""
    import numpy as np

    import oracle

    h = oracle.decode_u16(w.dem_u16) if w.dem_u16 is not None else w.dem_f32
    _, t2, _ = oracle.normals(h, w.cell_size, want_slope=False)
    _, cells = oracle.release(t2, w.slope_lo_deg, w.slope_hi_deg)
    p = oracle.SimParams(mu=w.mu, drag_k=w.drag_k, persistence=w.persistence, randomness=w.randomness,
                         step_scale=w.step_scale, gravity=w.gravity, traj_per_cell=w.traj_per_cell,
                         max_steps=w.max_steps, seed=w.seed)
    threads = threads or os.cpu_count() or 1
    rng = np.random.default_rng(12345)
    rate = _oracle_rate(oracle, h, w.cell_size, cells, p, threads, rng)
    k = int(min(cells.size, max(threads, rate * seconds)))
    sample = np.sort(rng.choice(cells, k, replace=False))
    t0 = time.perf_counter()
    _, _, st = oracle.simulate_threaded(h, w.cell_size, sample, p, threads=threads, merge=False)
    dt = time.perf_counter() - t0
    return {"value": st["total_steps"] / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{k} of {cells.size} release cells (uniform random, seed 12345), all "
                       f"{w.traj_per_cell} particles each: {st['n_traj']} particles, {st['total_steps']} moves "
                       f"in {dt:.2f} s on {threads} threads"),
            "particles_per_s": st["n_traj"] / dt, "seconds": dt}


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------
def run_awo(args, R: Ranks):
    import numpy as np
    import torch

    import paper_2506_23364_gb300 as awo

    w = _workload(args.workload, args.crop)
    params = awo.SimParams.make(mu=w.mu, drag_k=w.drag_k, persistence=w.persistence, randomness=w.randomness,
                                step_scale=w.step_scale, gravity=w.gravity, traj_per_cell=w.traj_per_cell,
                                max_steps=w.max_steps, seed=w.seed)
    ov = awo.Overlay(w.width, w.height, w.cell_size, quantised=w.quantised, levels=w.lod_levels,
                     device=R.device, want_slope=False, release_log2=args.release_log2)
    host_dem = w.dem_u16 if w.quantised else w.dem_f32
    ov.load_dem(host_dem)
    torch.cuda.synchronize()
    lo, hi = w.slope_lo_deg, w.slope_hi_deg

    def step(ev=None, kev=None):
        ov.terrain(lo, hi)
        if ev is not None:
            ev[0].record()
        if kev is not None:  # the particle kernel alone (not the output clear or the prologue)
            awo.awo_simulate_time_kernel(kev[0], kev[1])
        ov.simulate(params)
        if ev is not None:
            ev[1].record()
        ov.overlay(w.gravity)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st = ov.stats_dict()
    visits = st["total_steps"] + st["n_traj"]
    # decode and normals (one launch), release (mask, scan, scatter), particle prologue and kernel, then
    # velocity and mipmap: one launch for both and levels 1..6, one per further level (velocity alone
    # without a mipmap)
    lod_launches = 1 if w.lod_levels <= 1 else 1 + max(w.lod_levels - 1 - 6, 0)
    launches_per_step = 1 + 3 + 2 + lod_launches

    peaks_probe = _probe_peaks(torch, awo)
    clocks = ClockSampler(R.local)
    sim_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in kern_ev:  # create the events (torch makes them at their first record)
        a_.record()
        b_.record()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    R.barrier()
    torch.cuda.synchronize()
    t0.record()
    for k in range(args.steps):
        step(sim_ev[k], kern_ev[k])
    t1.record()
    torch.cuda.synchronize()
    R.barrier()
    clk = clocks.stop()
    ms_step = t0.elapsed_time(t1) / args.steps
    sim_ms = statistics.mean(a.elapsed_time(b) for a, b in sim_ev)  # awo_simulate: clear, prologue, kernel
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in kern_ev)  # the particle kernel alone
    st2 = ov.stats_dict()
    assert st2 == st, "particle statistics changed between runs"
    ms_step_max = R.reduce(ms_step, "max")
    total_steps_all = R.reduce(float(st["total_steps"]), "sum")
    value = total_steps_all / (ms_step_max / 1e3)

    # end to end through the API with host buffers: H2D of the DEM, D2H of the overlay (all levels)
    e2e = _e2e(args, R, awo, w, ov, host_dem, lambda o: o.terrain(lo, hi),
               lambda o: (o.simulate(params), o.overlay(w.gravity)),
               float(st["total_steps"]), total_steps_all)

    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sim_s = kern_ms / 1e3  # roofline denominators: the particle kernel's own launch
    sha = _kernel_sha()
    # the counters are per visit of the 8192^2 workload's launch (its 6144^2 crop): other workloads (the
    # long-trajectory ones, a release texture) visit differently, so they report none
    same_launch = args.workload == "large" and not args.release_log2
    kc = KERNEL_COUNTERS.get(sha, {}) if same_launch else {}
    traffic = kc.get("dram")
    # issue / ALU ceiling: 152 SMs x 128 lanes x SM clock (max clock of the run)
    sms = torch.cuda.get_device_properties(R.device).multi_processor_count
    mhz = clk.get("sm_max_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * mhz * 1e6 / 1e12
    alu_achieved = ALG_OPS_PER_VISIT * visits / sim_s / 1e12
    roofline = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": alu_achieved / alu_peak,
                "traffic": traffic * visits if traffic is not None else None, "kernel": "k_simulate",
                "kernel_ms": kern_ms, "units_per_launch": visits, "alg_ops_per_unit": ALG_OPS_PER_VISIT,
                "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz (issue ceiling; ncu: issue-bound)"}
    alg_bytes = ALG_BYTES_PER_VISIT * visits
    roofline_hbm = {"achieved": alg_bytes / sim_s / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": alg_bytes / sim_s / 1e9 / hbm, "alg_bytes_per_launch": alg_bytes,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}
    # L2: the hardware's own utilisation of the L2 for this kernel (ncu), the
    # gather/reduction roofline fraction; sector rates beside it
    l2 = {"frac": kc.get("lts_frac"), "source": ("ncu lts__throughput.avg.pct_of_peak_sustained_elapsed, "
                                                 "6144^2 crop launch of the same kernel code") if same_launch else
                                                ("none: the counters were taken on the 8192^2 workload "
                                                 "(ncu figures for this workload are in the profiles)"),
          "reduction_units_busy": kc.get("atomic_busy"),
          "red_sector_ops_per_s": kc["red_sectors"] * visits / sim_s if kc else None,
          "read_sectors_per_s": kc["read_sectors"] * visits / sim_s if kc else None,
          "random_access_probe": {"l2_red_per_s": peaks_probe["l2_red_per_s"],
                                  "l2_load_per_s": peaks_probe["l2_gather_per_s"],
                                  "note": "per-lane hashed 4-byte accesses (one sector each); context, not a "
                                          "ceiling: the kernel's lanes share sectors"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": R.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded fBm + carved valleys, uint16 dm)",
            "config": dict(w.describe(), parallelism=f"replicas x{R.world}" if R.world > 1 else "single GPU",
                           l2="inputs larger than L2 (uint16 DEM 128 MiB + FP32 DEM 256 MiB + rasters)",
                           release_cells=ov.n_release(), **({"release_texture_log2": args.release_log2,
                                                             "release_texture": [ov.g_rel.width, ov.g_rel.height]}
                                                            if args.release_log2 else {})),
            "ms_per_overlay": ms_step_max, "simulate_ms": sim_ms,
            "simulate_steps_per_s": st["total_steps"] / (sim_ms / 1e3),
            "particles_per_s": st["n_traj"] / (sim_ms / 1e3), "stats": st,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "roofline": roofline, "roofline_l2": l2,
            "roofline_hbm": roofline_hbm,
            "clocks": clk, "kernel_sha": sha}
    if R.rank == 0 and R.world == 1 and not args.no_cpu_baseline and not args.release_log2:
        line["cpu_baseline"] = _cpu_baseline(w, args.cpu_seconds, args.cpu_threads or None)
    if (R.world == 1 and args.workload == "large" and not args.crop and not args.release_log2
            and not args.no_extensions):
        line["extensions"] = _extensions(args, R)
    if R.rank == 0:
        print(json.dumps(line), flush=True)


def _extensions(args, R: Ranks) -> dict:
    """Compact runs of the batched, served, differentiable and parabola
    workloads (each function's own measurement, fewer steps), reported
    beside the headline so that they are measured in the same run."""
    import torch

    keep = {"batched": ("value", "unit", "ms_per_step", "speedup_vs_plain", "rasters_equal_plain", "alu", "clocks"),
            "served": ("value", "unit", "latency_ms", "ok", "mean_batch", "wall_s", "clocks"),
            "differentiable": ("forward_ms", "backward_ms", "particles", "moves", "fd_rel_err"),
            "parabola": ("value", "unit", "min_ms", "particles", "moves")}
    out = {}
    for name, fn, steps in (("batched", run_batched, 3), ("served", run_served, args.steps),
                            ("differentiable", run_diff, 3), ("parabola", run_parabola, 10)):
        a = argparse.Namespace(**vars(args))
        a.steps, a.warmup = steps, 1
        t0 = time.perf_counter()
        try:
            r = fn(a, R, emit=False)
        except Exception as e:  # reported, not hidden: the headline line still prints
            out[name] = {"error": repr(e)[:400]}
            continue
        d = {k: r[k] for k in keep[name] if k in r}
        d["config"] = r.get("config", {}).get("workload")
        if name == "batched":
            d["plain_value"] = r["plain"]["value"]
            d["regions_by_texture_gather"] = r["config"].get("regions_by_texture_gather")
        d["wall_s"] = d.get("wall_s") or (time.perf_counter() - t0)
        out[name] = d
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def _e2e(args, R, awo, w, ov, host_dem, terrain, particles, steps_one, steps_all) -> dict:
    """The same workload end to end through the public API: every step copies
    its DEM from pinned host memory, runs the workflow (terrain(o), then
    particles(o): the particle run with its velocity and mipmap) and copies
    the whole overlay (count and velocity, every mipmap level) back to pinned
    host memory.  Pipelined form (the value): --e2e-instances workflow
    instances (default 3) on as many CUDA streams take steps in turn, so the
    copies of one step overlap the kernels of the next; 4 x --e2e-steps steps
    are timed so that the unoverlapped first copy-in and last copy-out weigh
    little.  The particle run of step k waits for the mipmap pass of step
    k - 2: the particle kernel is persistent (it holds every SM until its
    work runs out), so a mipmap pass that became ready behind two of them
    would hold its step's copy-out, and with it a later step, for two whole
    particle runs; neighbouring steps' particle kernels still share their
    tails.  Serial form (reported beside it): one stream, each step
    synchronised before the next."""
    import numpy as np
    import torch

    src = np.ascontiguousarray(host_dem).view(np.int16) if w.quantised else host_dem
    pin_dem = torch.from_numpy(src).pin_memory()
    m = max(1, args.e2e_instances)
    extra = [awo.Overlay(w.width, w.height, w.cell_size, quantised=w.quantised, levels=w.lod_levels,
                         device=R.device, want_slope=False, release_log2=ov.release_log2) for _ in range(m - 1)]

    def outs_of(o):
        dev = [o.count, o.vel] + [t for pair in zip(o.count_lv, o.vel_lv) for t in pair]
        return [(d, torch.empty(d.shape, dtype=d.dtype).pin_memory()) for d in dev]

    insts = [(o, outs_of(o), torch.cuda.Stream(R.device)) for o in [ov] + extra]
    bi = pin_dem.numel() * pin_dem.element_size()
    bo = sum(h.numel() * h.element_size() for _, h in insts[0][1])

    def one(inst, after=None):
        o, outs, s = inst
        with torch.cuda.stream(s):
            (o.q if w.quantised else o.h).copy_(pin_dem, non_blocking=True)
            terrain(o)
            if after is not None:
                s.wait_event(after)
            particles(o)
            done = torch.cuda.Event()
            done.record(s)
            for d, h in outs:
                h.copy_(d, non_blocking=True)
        return done

    n = max(args.e2e_steps, 1)
    # serial: one instance, synchronised per step
    serial = []
    for k in range(n + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        R.barrier()
        a.record(insts[0][2])
        one(insts[0])
        b.record(insts[0][2])
        b.synchronize()
        if k > 0:
            serial.append(a.elapsed_time(b))
    serial_ms = R.reduce(statistics.mean(serial), "max")
    # pipelined: m instances on m streams, one warm-up step each, then 4 n steps
    for inst in insts:
        one(inst)
    torch.cuda.synchronize()
    R.barrier()
    s0 = insts[0][2]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s0)
    for inst in insts[1:]:
        inst[2].wait_event(a)
    k_steps = 4 * n
    lag = 2  # the particle run of step k waits for the mipmap pass of step k - lag
    dones = []
    for k in range(k_steps):
        dones.append(one(insts[k % m], dones[k - lag] if k >= lag else None))
    for inst in insts[1:]:
        s0.wait_stream(inst[2])
    b.record(s0)
    b.synchronize()
    pipe_ms = R.reduce(a.elapsed_time(b) / k_steps, "max")
    del extra, insts
    return {"value": steps_all / (pipe_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "ms_per_step": pipe_ms, "steps": k_steps,
            "form": f"{m} workflow instances on {m} CUDA streams, steps in turn (copies overlap the next step; "
                    f"step k's particle run after step k - {lag}'s mipmap pass)",
            "serial": {"value": steps_all / (serial_ms / 1e3), "ms_per_step": serial_ms, "steps": n,
                       "form": "1 stream, synchronised after every step"}}


def _region_params(awo, r):
    return awo.SimParams.make(**r.params)


def run_batched(args, R: Ranks, emit: bool = True) -> dict:
    """Many regions: each region run alone in sequence (the plain form) against
    one batched launch per pass (tuned once, replayed from a CUDA graph)."""
    import torch

    import paper_2506_23364_gb300 as awo
    from paper_2506_23364_gb300 import inputs

    reqs = inputs.batched_requests(args.batch_n)
    params = [_region_params(awo, r) for r in reqs]
    cs = reqs[0].cell_size
    ovs = []
    for r in reqs:
        H, W = r.dem_u16.shape
        ov = awo.Overlay(W, H, cs, quantised=True, levels=1, device=R.device, want_normals=False, want_mask=False)
        ov.load_dem(r.dem_u16)
        ovs.append(ov)

    def plain():
        for ov, r, p in zip(ovs, reqs, params):
            ov.run(*r.release_deg, p)

    def timed(fn, k):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / k

    ms_plain = timed(plain, args.steps)
    steps_plain = sum(ov.stats_dict()["total_steps"] for ov in ovs)
    batch = awo.Batch([r.dem_u16 for r in reqs], cs, params, [r.release_deg for r in reqs], quantised=True,
                      device=R.device)
    tuning, tune_ms = batch.tune()
    batch.capture()
    clocks = ClockSampler(R.local)
    clocks.start()
    ms_batch = timed(batch.replay, args.steps)
    clk = clocks.stop()
    st = batch.stats_list()
    steps_batch = sum(x["total_steps"] for x in st)
    assert steps_batch == steps_plain, "batched and plain runs must make the same moves"
    # every region's rasters and statistics from the graph replay against its plain run, on the device
    same = all(torch.equal(bo.count, po.count) and torch.equal(bo.maxe, po.maxe) and torch.equal(bo.vel, po.vel)
               and x == po.stats_dict() for bo, po, x in zip(batch.ovs, ovs, st))
    assert same, "batched rasters differ from the plain runs"
    paths = [awo.awo_dem_gather_path(ov.h, ov.g) for ov in batch.ovs]
    del ovs
    cells = sum(r.dem_u16.size for r in reqs)
    line = {"metric": "aggregate trajectory-steps/s, batched regions", "value": steps_batch / (ms_batch / 1e3),
            "unit": UNIT, "n_gpus": R.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded fBm regions, uint16 dm)",
            "config": {"workload": f"batched-{len(reqs)}-regions-512..4096", "cells": cells,
                       "particles": sum(x["n_traj"] for x in st), "form": "one batched launch per pass, CUDA graph",
                       "tuning": tuning.as_dict(), "tune_best_ms": tune_ms,
                       "regions_by_texture_gather": paths.count("texture")},
            "rasters_equal_plain": same,
            "plain": {"value": steps_plain / (ms_plain / 1e3), "ms_per_pass": ms_plain,
                      "form": "each region alone, in sequence, same stream"},
            "speedup_vs_plain": ms_plain / ms_batch, "clocks": clk}
    # the particle kernels' ALU/issue count over the whole pass (terrain,
    # prologues and mipmaps of the 64 regions included, so a lower bound)
    sms = torch.cuda.get_device_properties(R.device).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    visits = steps_batch + sum(x["n_traj"] for x in st)
    line["alu"] = {"frac_whole_pass": ALG_OPS_PER_VISIT * visits / (ms_batch / 1e3) / (sms * 128 * mhz * 1e6),
                   "visits": visits, "alg_ops_per_unit": ALG_OPS_PER_VISIT,
                   "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz"}
    if emit and R.rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_served(args, R: Ranks, emit: bool = True) -> dict:
    """Poisson arrivals of the batched workload's regions into the serving loop."""
    import torch

    from paper_2506_23364_gb300 import inputs
    from paper_2506_23364_gb300.serve import OverlayRequest, OverlayServer, latency_summary

    regs = inputs.batched_requests(args.batch_n)
    mk = lambda r: OverlayRequest(r.dem_u16, r.cell_size, r.release_deg, dict(r.params))
    srv = OverlayServer(budget_bytes=96 << 30, n_slots=4, max_batch=16, device=R.device)
    for f in [srv.submit(mk(r)) for r in regs[:4]]:  # warm-up (library load, occupancy queries, allocator)
        f.result()
    arrivals = inputs.poisson_arrivals(len(regs), args.rate, seed=1)
    clocks = ClockSampler(R.local)
    clocks.start()
    t0 = time.perf_counter()
    futs = []
    for r, at in zip(regs, arrivals):
        dt = t0 + at - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        futs.append(srv.submit(mk(r)))
    res = [f.result() for f in futs]
    t_end = max(x.t_done for x in res)
    clk = clocks.stop()
    srv.shutdown()
    ok = [x for x in res if x.status == "ok"]
    steps = sum(x.stats["total_steps"] for x in ok)
    lat = latency_summary(res)
    line = {"metric": "served overlays: p50/p99 latency and aggregate trajectory-steps/s",
            "value": steps / (t_end - t0), "unit": UNIT, "n_gpus": R.world, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic (seeded fBm regions, uint16 dm)",
            "config": {"workload": f"served-{len(regs)}-regions-512..4096", "arrivals": f"Poisson {args.rate}/s",
                       "slots": 4, "max_batch": 16, "budget_gib": 96},
            "latency_ms": lat, "ok": len(ok), "mean_batch": float(np.mean([x.batch_size for x in ok])),
            "wall_s": t_end - t0, "peak_budget_gib": srv.sched.peak_in_use / 2 ** 30, "clocks": clk}
    if emit and R.rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_diff(args, R: Ranks, emit: bool = True) -> dict:
    """Differentiable workload: soft deposits on a 1024^2 fBm DEM, target at
    hidden friction parameters, L2 loss; forward and adjoint timed with CUDA
    events; the gradient checked against central differences (h = 1e-3)."""
    import torch

    import paper_2506_23364_gb300 as awo
    from paper_2506_23364_gb300 import inputs

    n = 1024
    dem = inputs.quantise_dm(inputs.fbm(n, 0.8, seed=3, relief=3000.0 * (n / 2048.0) ** 0.8))
    prob = awo.SoftOverlay(dem, inputs.CELL_SIZE_M, inputs.MID_RELEASE_DEG, traj_per_cell=128, max_steps=2048,
                           seed=0, device=R.device)
    w = torch.from_numpy(np.random.default_rng(3).uniform(0.5, 1.5, prob.n_cells).astype(np.float32)).to(R.device)
    mu0, k0 = float(np.tan(np.deg2rad(25.0))), 1e-3
    Dstar = prob.forward_raw(mu0 * 1.2, k0 * 0.8, w)
    loss = lambda mu, k: float(((prob.forward_raw(mu, k, w) - Dstar) ** 2).sum())
    fwd, bwd = [], []
    for it in range(args.warmup + args.steps):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        D = prob.forward_raw(mu0, k0, w)
        b.record()
        gt, gw = prob.backward_raw(mu0, k0, w, 2.0 * (D - Dstar))
        c.record()
        c.synchronize()
        if it >= args.warmup:
            fwd.append(a.elapsed_time(b))
            bwd.append(b.elapsed_time(c))
    g = gt.cpu().tolist()
    h = 1e-3
    fd = [(loss(mu0 * np.exp(h), k0) - loss(mu0 * np.exp(-h), k0)) / (2 * h),
          (loss(mu0, k0 * np.exp(h)) - loss(mu0, k0 * np.exp(-h))) / (2 * h)]
    st = prob.stats.cpu().tolist()
    line = {"metric": "differentiable soft-deposit overlay: forward + adjoint ms", "value":
            statistics.median(fwd) + statistics.median(bwd), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32 (f64 gradient reductions)",
            "data": "synthetic (seeded fBm, uint16 dm)",
            "config": {"workload": "diff-fbm-1024", "release_cells": prob.n_cells, "traj_per_cell": 128,
                       "max_steps": 2048, "theta_star": "(1.2 mu0, 0.8 k0)", "tau_m": prob.tau},
            "forward_ms": statistics.median(fwd), "backward_ms": statistics.median(bwd),
            "particles": st[1], "moves": st[0],
            "grad_log_mu": g[0], "grad_log_k": g[1], "fd_log_mu": fd[0], "fd_log_k": fd[1],
            "fd_rel_err": [abs(g[0] - fd[0]) / abs(fd[0]), abs(g[1] - fd[1]) / abs(fd[1])],
            "grad_w_norm": float(gw.norm())}
    if emit and R.rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_parabola(args, R: Ranks, emit: bool = True) -> dict:
    """Parabola-shaped stand-in (501 x 151, three given release cells, 2048
    particles each): the whole workflow per step, from the device-resident DEM
    and release mask."""
    import torch

    import paper_2506_23364_gb300 as awo
    from paper_2506_23364_gb300 import inputs

    w = inputs.parabola()
    ov = awo.Overlay(w.width, w.height, w.cell_size, quantised=False, levels=1, device=R.device)
    ov.load_dem(w.dem_f32)
    mask = torch.from_numpy(inputs.parabola_release_mask()).to(R.device)
    p = awo.SimParams.make(mu=w.mu, persistence=w.persistence, randomness=w.randomness,
                           traj_per_cell=w.traj_per_cell, max_steps=w.max_steps, seed=w.seed)

    def step():
        ov.terrain_from_mask(mask)
        ov.simulate(p)
        ov.overlay(w.gravity)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    st = ov.stats_dict()
    line = {"metric": "ms per overlay, parabola-shaped stand-in", "value": statistics.median(ts), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "data": "synthetic parabola-shaped slope (stand-in; the paper's dataset is not available)",
            "config": dict(w.describe(), release="3 given cells (mask)"),
            "vs_baseline": None, "context": "paper Table 1: weBIGeo 13.5 ms on an RTX 3070 (WebGPU) for its "
                                             "parabola dataset; different geometry and hardware",
            "particles": st["n_traj"], "moves": st["total_steps"], "min_ms": min(ts)}
    if emit and R.rank == 0:
        print(json.dumps(line), flush=True)
    return line


def run_stages(args, R: Ranks):
    """Each streaming (HBM-bound) stage alone on the 8192^2 workload's rasters,
    CUDA-event timed (median of --steps after --warmup), against the measured
    HBM copy bandwidth.  Algorithmic bytes are each stage's inputs read once
    and outputs written once (a release pass: tan^2 in, mask and list out)."""
    import torch

    import paper_2506_23364_gb300 as awo
    from paper_2506_23364_gb300 import inputs

    w = _workload("large", args.crop)
    ov = awo.Overlay(w.width, w.height, w.cell_size, quantised=True, levels=w.lod_levels, device=R.device,
                     want_slope=True)
    ov.load_dem(w.dem_u16)
    p = awo.SimParams.make(traj_per_cell=w.traj_per_cell, max_steps=w.max_steps)
    ov.run(w.slope_lo_deg, w.slope_hi_deg, p)
    torch.cuda.synchronize()
    n = w.width * w.height
    n_rel = ov.n_release()
    g = ov.g
    cm = awo.Colormap.make(awo.VELOCITY_STOPS, alpha=0.7, count_min=1)
    base = torch.zeros((w.height, w.width, 4), dtype=torch.uint8, device=R.device)
    rgba = torch.empty_like(base)
    alpha = torch.empty((w.height, w.width), dtype=torch.float32, device=R.device)
    sp = awo.SnowParams(1500.0, 300.0, 36.0, 4.0)
    nz = ov.normal[2]
    lv_bytes = sum(c.numel() * 8 for c in ov.count_lv)
    # release on the texture at 2x the DEM resolution (4 texels per cell)
    wr, hr = awo.awo_release_texture_dims(g, 1)
    mask_t = torch.empty(wr * hr, dtype=torch.uint8, device=R.device)
    tex = torch.empty(wr * hr, dtype=torch.int32, device=R.device)
    n_tex = torch.zeros(1, dtype=torch.int32, device=R.device)
    ws_t = torch.empty(awo.awo_release_texture_workspace_bytes(g, 1), dtype=torch.uint8, device=R.device)

    def rel_tex():
        awo.awo_release_texture(ov.tan2, g, 1, w.slope_lo_deg, w.slope_hi_deg, mask_t, tex, n_tex, ws_t)

    rel_tex()
    torch.cuda.synchronize()
    n_rel_t = int(n_tex.item())
    stages = [
        ("decode", lambda: awo.awo_decode_u16(ov.q, g, 0.1, ov.h), 6 * n),
        ("normals (+tan2)", lambda: awo.awo_normals(ov.h, g, ov.normal, ov.tan2, None), 20 * n),
        ("normals (+tan2, slope_deg)", lambda: awo.awo_normals(ov.h, g, ov.normal, ov.tan2, ov.slope), 24 * n),
        ("decode + normals (one pass)", lambda: awo.awo_normals_u16(ov.q, g, 0.1, ov.h, ov.normal, ov.tan2, None),
         22 * n),
        ("release (3 passes)", lambda: awo.awo_release(ov.tan2, g, w.slope_lo_deg, w.slope_hi_deg, ov.mask, ov.cells,
                                                       ov.n_rel, ov.ws_rel), 5 * n + 4 * n_rel),
        ("release texture 2x (3 passes)", rel_tex, 4 * n + wr * hr + 4 * n_rel_t),
        ("finalize", lambda: awo.awo_finalize(ov.maxe, g, 9.81, ov.vel), 8 * n),
        ("mipmap (5 levels)", lambda: awo.awo_overlay_lod(ov.count, ov.vel, g, w.lod_levels, ov.count_lv, ov.vel_lv),
         8 * n + lv_bytes),
        ("finalize + mipmap (one pass)", lambda: awo.awo_finalize_lod(ov.maxe, ov.count, g, 9.81, w.lod_levels, ov.vel,
                                                                      ov.count_lv, ov.vel_lv), 12 * n + lv_bytes),
        ("compose over base", lambda: awo.awo_compose(ov.vel, ov.count, g, cm, base, rgba), 16 * n),
        ("snow cover (alpha + rgba)", lambda: awo.awo_snow_cover(ov.h, nz, g, sp, alpha, rgba), 16 * n),
    ]
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    rows = []
    for name, fn, nbytes in stages:
        for _ in range(max(args.warmup, 1)):
            fn()
        ts = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        gbs = nbytes / (ms / 1e3) / 1e9
        rows.append({"stage": name, "ms": ms, "alg_bytes": nbytes, "GB/s": gbs, "frac_hbm": gbs / hbm})
    line = {"metric": "streaming stages at 8192^2: GB/s of algorithmic bytes vs measured HBM copy bandwidth",
            "unit": "GB/s", "hbm_peak_gbs": hbm, "config": {"workload": w.name, "cells": n, "release_cells": n_rel,
                                                            "release_texels_2x": n_rel_t},
            "stages": rows}
    if R.rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, R: Ranks):
    """The CPU oracle on the host cores: each step a bounded random sample of
    the workload's release cells (all particles of each)."""
    if R.rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2506_23364_gb300 import inputs

    if args.workload not in ("large", "mid", "tiny", "parabola"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the large, mid, tiny and "
                                                               "parabola workloads"}), flush=True)
        return
    if args.workload == "parabola":
        w = inputs.parabola()
        h = w.dem_f32
        cells = np.flatnonzero(inputs.parabola_release_mask().ravel()).astype(np.uint32)
    else:
        w = _workload(args.workload, args.crop)
        h = oracle.decode_u16(w.dem_u16) if w.dem_u16 is not None else w.dem_f32
        _, t2, _ = oracle.normals(h, w.cell_size, want_slope=False)
        _, cells = oracle.release(t2, w.slope_lo_deg, w.slope_hi_deg)
    p = oracle.SimParams(mu=w.mu, drag_k=w.drag_k, persistence=w.persistence, randomness=w.randomness,
                         step_scale=w.step_scale, gravity=w.gravity, traj_per_cell=w.traj_per_cell,
                         max_steps=w.max_steps, seed=w.seed)
    threads = args.cpu_threads or os.cpu_count() or 1
    total = args.steps + max(args.warmup, 0)
    per_step_s = max(min(1.0, args.cpu_seconds), min(10.0, args.cpu_seconds, 150.0 / max(total, 1)))
    rng = np.random.default_rng(777)
    rate = _oracle_rate(oracle, h, w.cell_size, cells, p, threads, rng)
    k = int(min(cells.size, max(threads, rate * per_step_s)))
    steps_done, secs = 0, 0.0
    for s in range(total):
        sample = np.sort(rng.choice(cells, k, replace=False))
        t0 = time.perf_counter()
        _, _, st = oracle.simulate_threaded(h, w.cell_size, sample, p, threads=threads, merge=False)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            steps_done += st["total_steps"]
            secs += dt
    value = steps_done / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": R.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded fBm + carved valleys, uint16 dm)",
            "config": dict(w.describe(), parallelism="host cores"),
            "timed": (f"particle stage only (the oracle's trajectories), per step a uniform random sample of "
                      f"{k} of {cells.size} release cells ({k / cells.size:.3g} of them); the GPU arm times the "
                      f"whole workflow over every release cell"),
            "reference_sample_frac": k / cells.size,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"per step {k} of {cells.size} release cells, all {w.traj_per_cell} "
                                       f"particles each (uniform random, seed 777)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    R = Ranks()
    try:
        if args.impl == "reference":
            run_reference(args, R)
        elif args.workload == "batched":
            run_batched(args, R)
        elif args.workload == "served":
            run_served(args, R)
        elif args.workload == "diff":
            run_diff(args, R)
        elif args.workload == "parabola":
            run_parabola(args, R)
        elif args.workload == "stages":
            run_stages(args, R)
        else:
            run_awo(args, R)
    finally:
        R.close()


if __name__ == "__main__":
    main()

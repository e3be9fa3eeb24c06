"""Benchmark of the adaptive PBF step on one GB300 (or N replicas).

Workload (default): 1,048,576 particles (128x128x64 block in a 9.6x6.4x4.8 m
basin with an oscillating wall, spline camera), APBF with N_i in 3..15 from
the distance to the camera, beside plain PBF with N = 15 on identical inputs.
A "step" is one simulation step of Fig. 7 (all stages) of that scene.

Metric: APBF ms/step (lower is better), with PBF(N_max) ms/step, the
performance improvement T_PBF/T_APBF - 1 (Table 1), p50/p99 step latency,
particle-iterations/s and the density error of both runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the scene (the single-scene
solver does not shard); rank 0 prints the JSON line with the max over ranks.
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

from paper_1608_04721_gb300 import metrics, scenes  # noqa: E402

METRIC = "APBF ms/step @1M particles vs PBF N_max, same GPU & density error; p50/p99 latency"
UNIT = "ms/step"
FP32_LANES_PER_SM = 128
SMS = 152
SM_MAX_MHZ = 2070.0
# algorithmic FP32 operations per in-range neighbour pair, the hot-path scope's
# figures: lambda ~30 (difference, r^2, poly6, spiky, the gradient and |grad|^2
# sums), delta-p ~35 plus one sqrt (spiky, poly6 for s_corr, its 4th power, the
# scaled vector sum); XSPH counted as in the kernel table (difference, r^2, W,
# neighbour velocity, difference x W, sum)
FLOPS_PER_PAIR = {"lambda": 30, "deltap": 36, "finalize": 26}
# algorithmic bytes per unit of the HBM-bound stages (each distinct array
# element read or written once per launch): unit "particle" or "cell"
STAGE_BYTES = {
    "predict": (40, "particle", "x, v read (32 B); key, slot written (8 B); the camera-distance range reduced on chip"),
    "scan": (12, "cell", "counts read, starts written, counts zeroed"),
    "scatter": (16, "particle", "key, slot read; start gathered; id written"),
    "reorder": (102, "particle", "44 B read (x, v, id, key, start); 58 B written (records, x*, ids, cells, "
                                 "levels in both orders)"),
    "levels": (8, "entry", "per (level bin, tile of 256 sorted slots): count read, offset written (the counts come "
                           "from the reorder pass; the neighbour search places the particles)"),
    "finalize": (76, "particle", "records, start positions read; x, v, id written (own particle; "
                                 "neighbour records via cache)"),
}
# per-step device state of one scene, for the L2 decision (neighbour lists at
# 128 entries dominate): an estimate shared by both arms of the benchmark
STATE_BYTES_PER_PARTICLE = 660
STAGE_NAMES = ["depth_image", "predict", "scan", "scatter", "reorder", "neighbors", "levels", "lambda", "deltap",
               "finalize", "prestab"]


DTVS_VIEW = (1280, 720, math.tan(math.radians(30.0)), (0.0, 0.0, 1.0))  # width, height, tan(fov_y/2), up


def workload(name: str, lod: str):
    if name == "ocean_1m":
        cfg = scenes.config_ocean_1m()
    elif name == "dam_break_131k":
        cfg = scenes.config_dam_break_131k()
    elif name == "multi_dam_break_225k":
        cfg = scenes.config_multi_dam_break_225k()
    elif name == "dam_break_4k":
        cfg = scenes.config_dam_break_4k().replace(lod_mode=scenes.LOD_DTC, n_min=2, n_max=4, camera="fixed",
                                                   eye=(-1.0, 0.8, 0.8))
    else:
        raise SystemExit(f"unknown workload {name}")
    if lod == "pbf":
        cfg = cfg.replace(lod_mode=scenes.LOD_FIXED, n_min=cfg.n_max)
    elif lod == "pbf_nmin":
        cfg = cfg.replace(lod_mode=scenes.LOD_FIXED, n_max=cfg.n_min, stabil_s=1)
    elif lod == "dtvs":
        cfg = cfg.replace(lod_mode=scenes.LOD_DTVS)
    return cfg


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    """Host-side process group (gloo) for barriers and the max over ranks;
    the data path has no collective."""

    def __init__(self):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as td

            td.init_process_group(backend="gloo")
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        return self.reduce(x, "max")

    def sum(self, x: float) -> float:
        return self.reduce(x, "sum")

    def reduce(self, x: float, op: str) -> float:
        if not self.pg:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(num(r[3]) for r in rows)}


def kernels_per_step(cfg) -> int:
    """Kernel launches of one step of a distance-to-camera (or fixed-level) scene."""
    k = 1 + 2 + 1 + 1 + 1 + 1  # predict (with the distance range), scan (2), scatter, reorder, neighbors, finalize
    if cfg.lod_mode != scenes.LOD_FIXED and cfg.n_max > cfg.n_min:
        k += 1  # level scan (the per-tile counts come from the reorder pass, the placement from the neighbour search)
    if getattr(cfg, "stabil_s", 0) > 1 and getattr(cfg, "stabil_iters", 0) > 0:
        k += 1  # pre-stabilisation
    return k + 2 * cfg.n_max


def make_scene(apbf, cfg, rho0, stream=None):
    x, v = scenes.make_scene(cfg)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, rho0), stream=stream)
    if cfg.obstacles:
        apbf.apbf_set_obstacles(s, cfg.obstacles)
    if cfg.lod_mode == scenes.LOD_DTVS:
        W, H, t, up = DTVS_VIEW
        drive(apbf, s, cfg, 0)
        apbf.apbf_set_view(s, W, H, t, up, 0.5 * cfg.spacing)
    return s


def drive(apbf, scene, cfg, step):
    eye, d = scenes.camera_at(cfg, step)
    lo, hi = scenes.box_at(cfg, step)
    apbf.apbf_set_camera(scene, eye, d)
    apbf.apbf_set_box(scene, lo, hi)


L2_BYTES = 129 * 2 ** 20
_flush_buf = None


def needs_flush(n_particles: int) -> bool:
    """A scene whose per-step state is below 4x the L2 could be served from L2
    across steps; such scenes are timed step by step with an L2 flush in between."""
    return n_particles * STATE_BYTES_PER_PARTICLE < 4 * L2_BYTES


def l2_note(n_particles: int) -> str:
    if needs_flush(n_particles):
        return ("flushed between timed steps (4x L2 written outside the timed intervals): per-step state "
                f"~{n_particles * STATE_BYTES_PER_PARTICLE / 1e6:.0f} MB")
    return (f"no flush: per-step state ~{n_particles * STATE_BYTES_PER_PARTICLE / 1e6:.0f} MB, over 4x the "
            "129 MB L2")


def workload_config(cfg, pbf_n: int, ws: int) -> dict:
    """The `config` of the JSON line, identical for the CUDA arm and the
    reference (oracle) arm of the same workload."""
    return {"workload": cfg.name, "particles": cfg.n, "n_range": f"{cfg.n_min}..{cfg.n_max}",
            "lod": "distance to camera, automatic range", "pbf_n": pbf_n,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU", "l2": l2_note(cfg.n)}


def flush_l2(torch):
    global _flush_buf
    if _flush_buf is None:
        _flush_buf = torch.empty(4 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    _flush_buf.fill_(1.0)


def timed_run(apbf, torch, scene, cfg, warmup, steps, first_step=0, flush=False):
    """Warm-up, then `steps` steps bracketed by CUDA events on the scene's
    stream; returns (total ms, per-step ms list, next step index). With
    flush, every timed step has its own pair of events and a write of 4x the
    L2 size runs between steps, outside the timed intervals."""
    stream = torch.cuda.current_stream()
    s = first_step
    for _ in range(warmup):
        drive(apbf, scene, cfg, s)
        apbf.apbf_step(scene, 1)
        s += 1
    apbf.apbf_sync(scene)
    torch.cuda.synchronize()
    if flush:
        a = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        z = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            drive(apbf, scene, cfg, s)
            flush_l2(torch)
            a[k].record(stream)
            apbf.apbf_step(scene, 1)
            z[k].record(stream)
            s += 1
        torch.cuda.synchronize()
        apbf.apbf_sync(scene)
        per = [a[k].elapsed_time(z[k]) for k in range(steps)]
        return sum(per), per, s
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        drive(apbf, scene, cfg, s)
        apbf.apbf_step(scene, 1)
        evs[k + 1].record(stream)
        s += 1
    torch.cuda.synchronize()
    apbf.apbf_sync(scene)
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return evs[0].elapsed_time(evs[-1]), per, s


def stage_profile(apbf, scene, cfg, first_step, steps, drive_fn=None):
    """Per-stage CUDA-event times over `steps` eager steps, plus the neighbour
    pairs each step's solver passes visited."""
    apbf.apbf_set_timing(scene, True)
    apbf.apbf_timing_report(scene)  # reset
    pairs = 0
    nbr_pairs = 0
    iters = 0
    ms_tot = np.zeros(len(STAGE_NAMES))
    ln_tot = np.zeros(len(STAGE_NAMES))
    s = first_step
    for _ in range(steps):
        (drive_fn or drive)(apbf, scene, cfg, s)
        apbf.apbf_step(scene, 1)
        info = apbf.apbf_get_step_info(scene)
        pairs += info["lambda_pairs"]
        nbr_pairs += info["neighbor_pairs"]
        iters += info["particle_iterations"]
        ms, ln = apbf.apbf_timing_report(scene)
        ms_tot += ms
        ln_tot += ln
        s += 1
    apbf.apbf_set_timing(scene, False)
    return ms_tot, ln_tot, pairs, nbr_pairs, iters, s


# What bounds the solver passes, from the committed ncu summary (not measured
# by this run): the roofline fraction above is against the FP32 pipes.
LIMITER_NOTE = ("L1 throughput: ncu puts the dense solver passes at 90 % (lambda) and 83 % (delta-p) of the L1 "
                "peak (warp-level gathers of 16-byte neighbour records, 19.5 sectors per request), DRAM at "
                "36-38 %, issue at 61-67 %, the FMA pipe at 42-46 % "
                "(profiles/solver_kernels_apbf_ocean_1048576.md)")


def hbm_peak():
    """(GB/s, source) from the measured peaks file, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy kernel)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no measured peak found)"


def copy_us(torch, nbytes: int, reps: int = 50) -> float:
    """CUDA-event time (us) of one device-to-device copy that moves nbytes in
    total (nbytes / 2 read, nbytes / 2 written), averaged over reps back-to-back
    copies: what a kernel of that size costs at best, launch included."""
    half = max(16, (nbytes // 2 + 15) // 16 * 16)
    src = torch.empty(half, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(src)
    for _ in range(3):
        dst.copy_(src)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        dst.copy_(src)
    z.record()
    torch.cuda.synchronize()
    return 1e3 * a.elapsed_time(z) / reps


def level_entries(cfg) -> int:
    """(level bin, tile) entries of the active-set partition: K bins x the
    tiles of 256 sorted slots, rounded up to a multiple of 4 (0 without one)."""
    if cfg.lod_mode == scenes.LOD_FIXED or cfg.n_max <= cfg.n_min:
        return 0
    return (cfg.n_max - cfg.n_min + 1) * (((cfg.n + 255) // 256 + 3) // 4 * 4)


def stage_roofline(stage_ms: dict, n_particles: int, n_cells: int, torch=None, n_entries: int = 0) -> dict:
    """Achieved HBM fraction of each HBM-bound stage: its algorithmic bytes per
    step (STAGE_BYTES x particles or cells) over its CUDA-event time per step.
    With torch, each stage also gets the time of a device copy moving the same
    bytes (copy_us) and its own time's fraction of that (frac_of_copy): stages
    of a few MB are bound by a launch's ramp and tail, which the copy pays too."""
    peak, src = hbm_peak()
    out = {"peak_gbs": peak, "peak_source": src, "stages": {}}
    for name, (bpu, unit, what) in STAGE_BYTES.items():
        t = stage_ms.get(name, 0.0)
        if t <= 0.0:
            continue
        units = {"particle": n_particles, "cell": n_cells, "entry": n_entries}[unit]
        if units <= 0:
            continue
        gbs = bpu * units / (t * 1e-3) / 1e9
        out["stages"][name] = {"bytes_per_" + unit: bpu, "units": units, "us_per_step": t * 1e3,
                               "achieved_gbs": gbs, "frac": gbs / peak, "bytes": what}
        if torch is not None:
            c = copy_us(torch, bpu * units)
            out["stages"][name].update({"copy_us": c, "frac_of_copy": c / (t * 1e3)})
    return out


def kernel_source_digest(src: str | None = None) -> str:
    """First 16 hex digits of the sha256 of kernels.cu (or of the source text
    given) without its comments and blank lines: a change to the code
    invalidates a traffic capture, a change to a comment does not."""
    if src is None:
        src = open(os.path.join(ROOT, "paper_1608_04721_gb300", "csrc", "kernels.cu"), encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def read_traffic(kernel: str, workload_name: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload_name}.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_source_digest()
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == kernel and not ln.startswith("#"):
            kv = dict(p.split("=", 1) for p in parts[1:] if "=" in p)
            if kv.get("source") == digest:
                return float(kv["dram_bytes_per_launch"])
    return None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_step_ms(oracle, cfg, rho0, step: int, threads: int, x=None, v=None, ids=None):
    """One oracle step of the whole workload at the given thread count; the
    camera and wall of the given step. Returns (ms, threads used, state)."""
    used = oracle.set_threads(threads)
    if x is None:
        x, v = scenes.make_scene(cfg)
    eye, _ = scenes.camera_at(cfg, step)
    lo, hi = scenes.box_at(cfg, step)
    p = oracle.make_params(cfg, rho0=rho0, eye=eye, box_lo=lo, box_hi=hi)
    t0 = time.perf_counter()
    st = oracle.step(p, x, v, ids)
    return (time.perf_counter() - t0) * 1e3, used, (st.x, st.v, st.ids)


def cpu_baseline(cfg):
    """The oracle as it stands on the host cores: one step of the whole
    workload (every particle, no extrapolation) on all cores, and one on a
    single thread."""
    import oracle

    rho0 = float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))
    ms_all, used, _ = oracle_step_ms(oracle, cfg, rho0, 0, host_cores())
    ms_one, _, _ = oracle_step_ms(oracle, cfg, rho0, 0, 1)
    oracle.set_threads(host_cores())
    return {"value": ms_all, "unit": UNIT, "cores": used, "kind": "oracle", "nproc": host_cores(),
            "sample": f"one oracle step of the whole workload ({cfg.n} particles, first step's camera and wall), "
                      f"OpenMP over particles on {used} threads",
            "single_thread": {"value": ms_one, "unit": UNIT, "cores": 1}}


def partition_scenes(sizes, ws: int):
    """Particle-balanced split of independent scenes over ws ranks: largest
    first, each to the rank with the fewest particles so far (ties to the
    lower rank). Returns each rank's scene indices, ascending. No scene is
    split and no data crosses ranks."""
    load = [0] * ws
    parts = [[] for _ in range(ws)]
    for k in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(ws), key=lambda r: (load[r], r))
        parts[r].append(k)
        load[r] += sizes[k]
    return [sorted(p) for p in parts]


def tune_summary(res):
    return {"block": res["block"], "mask_threshold": res["mask_threshold"], "trial_ms": res["ms_per_step"],
            "candidates": len(res["trials"])}


def run_batch(args, apbf, torch, d):
    """Batched multi-scene stepping: 256 independent dam breaks (sizes
    log-uniform in 2048..65536 particles, N_i in 4..8 by camera distance)
    stepped as one batch, one launch per stage over all scenes, against the
    same scenes stepped one at a time (one scene, one graph, per call).
    Under N ranks the 256 scenes are split by partition_scenes (whole scenes,
    particle-balanced): strong scaling, no collective on the data path."""
    all_cfgs = scenes.config_batch_256()
    mine = partition_scenes([c.n for c in all_cfgs], d.ws)[d.rank]
    cfgs = [all_cfgs[k] for k in mine]
    c0 = cfgs[0]
    rho0 = float(np.float32(apbf.apbf_rest_density(c0.h, c0.mass, c0.spacing)))
    descs = []
    for c in cfgs:
        x, v = scenes.make_scene(c)
        descs.append(apbf.desc_from_config(c, x, v, rho0))
    n_total = sum(c.n for c in cfgs)
    n_job = int(d.sum(n_total))
    batch = apbf.apbf_create_batch(descs)
    for k, c in enumerate(cfgs):
        apbf.apbf_set_camera_at(batch, k, c.eye)
    tuning = "defaults (block 256, compacted levels)"
    if not args.no_autotune:
        tuning = tune_summary(apbf.apbf_autotune(batch, 4))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def time_steps(step_fn, warmup, steps):
        for _ in range(warmup):
            step_fn()
        torch.cuda.synchronize()
        d.barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for k in range(steps):
            step_fn()
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        d.barrier()
        return evs[0].elapsed_time(evs[-1]), [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]

    clocks = ClockSampler(torch.cuda.current_device())
    tot, per = time_steps(lambda: apbf.apbf_step(batch, 1), args.warmup, args.steps)
    ms_step = d.max(tot / args.steps)
    density = apbf.apbf_density_stats(batch)
    # one at a time: the same scenes, each its own scene object and graph, same tuning
    singles = []
    for k, c in enumerate(cfgs):
        s = apbf.apbf_create_scene(descs[k])
        apbf.apbf_set_camera(s, c.eye)
        if isinstance(tuning, dict):
            apbf.apbf_set_tuning(s, tuning["block"], tuning["mask_threshold"])
        singles.append(s)

    def step_all():
        for s in singles:
            apbf.apbf_step(s, 1)

    single_steps = max(3, min(args.steps, 100))
    stot, sper = time_steps(step_all, args.warmup, single_steps)
    single_ms = d.max(stot / single_steps)
    for s in singles:
        apbf.apbf_destroy_scene(s)
    # end to end: step, then read every scene's positions into pinned host memory
    e2e = None
    if not args.no_e2e:
        host_pos = torch.empty((n_total, 3), dtype=torch.float32, pin_memory=True).numpy()
        bufs = [torch.empty((n_total, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        e2e_steps = max(3, min(args.steps, 100))
        for _ in range(args.warmup):
            apbf.apbf_step(batch, 1)
            apbf.apbf_read_state(batch, pos=host_pos, vel=False)
        d.barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            apbf.apbf_step(batch, 1)
            apbf.apbf_read_positions_async(batch, bufs[k % 2].data_ptr())
        apbf.apbf_sync(batch)
        e2e_ms = d.max((time.perf_counter() - t0) * 1e3 / e2e_steps)
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            apbf.apbf_step(batch, 1)
            apbf.apbf_read_state(batch, pos=host_pos, vel=False)
        sync_ms = d.max((time.perf_counter() - t0) * 1e3 / e2e_steps)
        e2e = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 12 * n_total,
               "what": "per step: apbf_step of the batch, apbf_read_positions_async of all positions of all scenes "
                       "into one of two pinned host buffers (the copy overlaps the next step), apbf_sync after the "
                       "last step; cameras and walls are fixed, so nothing is uploaded",
               "sync_value": sync_ms, "sync_what": "the same with apbf_read_state (synchronising) every step"}
    clock_info = clocks.stop()
    ms_st, ln_st, pairs, nbr_pairs, iters, _ = stage_profile(apbf, batch, c0, 0, args.profile_steps,
                                                             drive_fn=lambda *a: None)
    stage_ms = {STAGE_NAMES[k]: float(ms_st[k] / args.profile_steps) for k in range(len(STAGE_NAMES))}
    top = max(("lambda", "deltap"), key=lambda k: stage_ms[k])
    k_top = STAGE_NAMES.index(top)
    launches = max(1.0, float(ln_st[k_top]))
    avg_launch_s = ms_st[k_top] / launches * 1e-3
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = FLOPS_PER_PAIR[top] * pairs / launches / avg_launch_s / 1e12
    roofline = {"bound": "alu", "kernel": f"{top}_kernel", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                "traffic": read_traffic(f"{top}_kernel", "apbf_batch_256"),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz",
                "limiter": LIMITER_NOTE,
                "flops_per_pair": FLOPS_PER_PAIR[top], "pairs_per_launch": pairs / launches,
                "avg_launch_us": avg_launch_s * 1e6}
    per_step_iters = iters / args.profile_steps
    line = {
        "metric": "batched APBF ms/step for 256 independent scenes vs one at a time", "value": ms_step,
        "unit": UNIT, "n_gpus": d.ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "apbf_batch_256", "scenes": len(all_cfgs), "particles": n_job,
                   "scenes_on_rank0": len(cfgs), "particles_on_rank0": n_total,
                   "particles_per_scene": f"log-uniform {min(c.n for c in cfgs)}..{max(c.n for c in cfgs)}",
                   "n_range": f"{c0.n_min}..{c0.n_max}", "lod": "distance to camera, automatic range per scene",
                   "parallelism": (f"scenes split over {d.ws} ranks, particle-balanced" if d.ws > 1
                                   else "single GPU"),
                   "l2": "no flush: each step touches > 1 GB (> 129 MB L2)",
                   "launch": "one captured CUDA graph per batch step", "tuning": tuning},
        "p50_ms": metrics.percentile(per, 50), "p99_ms": metrics.percentile(per, 99),
        "one_at_a_time": {"ms_per_step": single_ms, "p50_ms": metrics.percentile(sper, 50),
                          "p99_ms": metrics.percentile(sper, 99), "steps": single_steps,
                          "speedup_of_batch": single_ms / ms_step,
                          "gpu_launches_per_step": len(cfgs) * kernels_per_step(c0)},
        "particle_iterations_per_step": per_step_iters,
        "particle_iterations_per_s": d.sum(per_step_iters / (ms_step * 1e-3)),
        "neighbor_pairs_per_step": nbr_pairs / args.profile_steps,
        "density": {"batch": [float(v) for v in density],
                    "fields": ["mean|rho/rho0-1|", "max|rho/rho0-1|", "mean(rho/rho0-1)", "mean max(0,rho/rho0-1)"]},
        "roofline": roofline, "stage_ms_per_step": stage_ms, "e2e": e2e,
        "gpu_launches": kernels_per_step(c0) * args.steps, "clocks": clock_info,
    }
    if d.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(cfgs, rho0)
    apbf.apbf_destroy_scene(batch)
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


SERVE_METRIC = "served APBF particle-steps/s, Poisson arrivals, budget-sized pool; queueing and latency"


def _pct(v, q):
    return metrics.percentile(v, q) if v else None


def serve_pooled(apbf, torch, temps, descs, arrivals, seconds, budget, max_particles, target_ms, warmup):
    """The serving loop on the wall clock for `seconds`: arrivals submitted as
    their time comes, one tick (one batched step of every resident scene) after
    another. Returns the run's statistics."""
    srv = apbf.apbf_server_create(descs[0], max_particles=max_particles, budget_bytes=budget,
                                  target_step_ms=target_ms)
    pool_bytes, cap_n, cap_c = apbf.apbf_server_bytes(descs[0], max_particles=max_particles, budget_bytes=budget,
                                                      target_step_ms=target_ms)
    for k in range(warmup):  # graph capture, first launches; then drain
        apbf.apbf_server_submit(srv, descs[k % len(descs)], temps[k % len(temps)].eye, 3, want_pos=False)
    while True:
        info = apbf.apbf_server_tick(srv)
        if info["resident_scenes"] == 0 and info["queued"] == 0:
            break
    iters0 = info["total_particle_iterations"]
    torch.cuda.synchronize()
    tick_start, infos, reqs = [], [], []
    ai = 0
    t0 = time.perf_counter()
    first_tick = None
    idle = True
    while True:
        now = time.perf_counter() - t0
        if now >= seconds:
            break
        if idle and (ai >= len(arrivals) or arrivals[ai][0] > now):
            # nothing resident or queued: wait for the next arrival instead of ticking empty
            time.sleep(min(seconds, arrivals[ai][0] if ai < len(arrivals) else seconds) - now)
            continue
        while ai < len(arrivals) and arrivals[ai][0] <= now:
            ta, k, steps = arrivals[ai]
            tk = apbf.apbf_server_submit(srv, descs[k], temps[k].eye, steps, want_pos=True, want_vel=False)
            reqs.append((tk, ta, k, steps))
            ai += 1
        tick_start.append(now)
        info = apbf.apbf_server_tick(srv)
        if first_tick is None:
            first_tick = info["tick"]
        infos.append(info)
        idle = info["resident_scenes"] == 0 and info["queued"] == 0
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    # one more tick collects the last step's device time and the iteration count; what it
    # admits or retires happened after the window and is not counted
    last = apbf.apbf_server_tick(srv)
    n_ticks = len(tick_start)
    stepped = [i["resident_particles"] for i in infos if i["resident_scenes"] > 0]
    step_ms = [infos[k + 1]["prev_step_ms"] for k in range(len(infos) - 1) if infos[k]["resident_scenes"] > 0]
    if infos and infos[-1]["resident_scenes"] > 0:
        step_ms.append(last["prev_step_ms"])
    timeline = []
    for sec in range(int(math.ceil(seconds))):
        ks = [k for k, t in enumerate(tick_start) if sec <= t < sec + 1]
        if ks:
            timeline.append([sec, len(ks), int(sum(infos[k]["resident_particles"] for k in ks)),
                             int(max(infos[k]["resident_particles"] for k in ks)),
                             int(max(infos[k]["resident_scenes"] for k in ks)), int(infos[ks[-1]]["queued"])])
    waits, lat, done, adm, h2d, d2h = [], [], 0, 0, 0, 0
    for tk, ta, k, steps in reqs:
        q = apbf.apbf_server_query(srv, tk)
        if q["state"] in (apbf.APBF_REQ_RESIDENT, apbf.APBF_REQ_DONE) and q["admit_tick"] - first_tick < n_ticks:
            adm += 1
            waits.append(tick_start[q["admit_tick"] - first_tick] - ta)
            h2d += 24 * temps[k].n
        if q["state"] == apbf.APBF_REQ_DONE and q["done_tick"] - first_tick < n_ticks:
            done += 1
            lat.append(tick_start[q["done_tick"] - first_tick] - ta)
            d2h += 12 * temps[k].n
            srv._outputs.pop(tk, None)
    iters = last["total_particle_iterations"] - iters0
    apbf.apbf_server_destroy(srv)
    ticks = len(stepped)
    return {"elapsed_s": elapsed, "particle_steps": float(sum(stepped)), "particle_iterations": float(iters),
            "particle_steps_per_s": sum(stepped) / elapsed, "particle_iterations_per_s": iters / elapsed,
            "ticks": ticks, "step_ms_p50": _pct(step_ms, 50), "step_ms_p99": _pct(step_ms, 99),
            "step_ms_max": max(step_ms) if step_ms else None,
            "pool_gb": pool_bytes / 1e9, "capacity_particles": cap_n, "capacity_cells": cap_c,
            "target_step_ms": target_ms or None,
            "resident_particles_mean": float(np.mean(stepped)) if stepped else 0.0,
            "resident_particles_max": int(max(stepped)) if stepped else 0,
            "resident_scenes_max": int(max(i["resident_scenes"] for i in infos)) if infos else 0,
            "particle_limit_last": infos[-1]["particle_limit"] if infos else None,
            "requests": {"submitted": len(reqs), "admitted": adm, "completed": done,
                         "queued_at_end": infos[-1]["queued"] if infos else 0,
                         "queue_wait_s_p50": _pct(waits, 50), "queue_wait_s_p99": _pct(waits, 99),
                         "latency_s_p50": _pct(lat, 50), "latency_s_p99": _pct(lat, 99)},
            "timeline": {"fields": ["second", "ticks", "particle_steps", "resident_particles_max",
                                    "resident_scenes_max", "queued_at_end"], "rows": timeline},
            "h2d_bytes": h2d, "d2h_bytes": d2h}


def serve_one_at_a_time(apbf, torch, temps, descs, arrivals, seconds):
    """The same arrivals served first in, first out, one scene at a time: each
    request gets its own scene (created on the device, stepped alone through
    its captured graph, read back, destroyed) before the next one starts."""
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    ai, queue = 0, []
    steps_done, iters, step_ms, waits, lat, done = 0, 0, [], [], [], 0
    while True:
        now = time.perf_counter() - t0
        if now >= seconds:
            break
        while ai < len(arrivals) and arrivals[ai][0] <= now:
            queue.append(arrivals[ai])
            ai += 1
        if not queue:
            time.sleep(min(seconds, arrivals[ai][0] if ai < len(arrivals) else seconds) - now)
            continue
        ta, k, steps = queue.pop(0)
        waits.append(now - ta)
        s = apbf.apbf_create_scene(descs[k])
        apbf.apbf_set_camera(s, temps[k].eye)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        ran = 0
        for j in range(steps):
            apbf.apbf_step(s, 1)
            evs[j + 1].record(stream)
            ran += 1
            if j % 16 == 15 and time.perf_counter() - t0 >= seconds:
                break
        out = apbf.apbf_read_state(s, pos=True, vel=False)
        torch.cuda.synchronize()
        step_ms += [evs[j].elapsed_time(evs[j + 1]) for j in range(ran)]
        iters += apbf.apbf_get_step_info(s)["total_particle_iterations"]
        apbf.apbf_destroy_scene(s)
        steps_done += ran * temps[k].n
        if ran == steps:
            done += 1
            lat.append(time.perf_counter() - t0 - ta)
        del out
    elapsed = time.perf_counter() - t0
    return {"elapsed_s": elapsed, "particle_steps": float(steps_done), "particle_iterations": float(iters),
            "particle_steps_per_s": steps_done / elapsed, "particle_iterations_per_s": iters / elapsed,
            "step_ms_p50": _pct(step_ms, 50), "step_ms_p99": _pct(step_ms, 99),
            "requests": {"submitted": ai, "completed": done, "queued_at_end": len(queue),
                         "queue_wait_s_p50": _pct(waits, 50), "queue_wait_s_p99": _pct(waits, 99),
                         "latency_s_p50": _pct(lat, 50), "latency_s_p99": _pct(lat, 99)}}


def run_serve(args, apbf, torch, d):
    """Served scenes: Poisson arrivals (200/s) of dam breaks with 4096..262144
    particles for 30..300 steps each (N_i in 5..10), admitted in arrival order
    into one pool sized from an HBM budget, every resident scene stepped once
    per tick, for the arrival window on the wall clock. The same trace runs
    three ways: the pool admitting while it has room, the pool admitting under
    a step-latency target, and first in, first out one scene at a time. Each
    rank serves its own arrivals."""
    temps = scenes.config_serve_templates()
    arrivals = scenes.serve_arrivals(seconds=args.serve_seconds, templates=len(temps), seed=1608_04721 + 11 * d.rank)
    c0 = temps[0]
    rho0 = float(np.float32(apbf.apbf_rest_density(c0.h, c0.mass, c0.spacing)))
    # the templates start at rest: no velocity arrays, so queued requests hold positions only
    descs = [apbf.desc_from_config(c, scenes.make_scene(c)[0], None, rho0) for c in temps]
    budget = int(args.serve_budget_gb * 1e9)
    d.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    pooled = serve_pooled(apbf, torch, temps, descs, arrivals, args.serve_seconds, budget, args.serve_max_particles,
                          0.0, args.warmup)
    targeted = None
    if args.serve_target_ms > 0:
        targeted = serve_pooled(apbf, torch, temps, descs, arrivals, args.serve_seconds, budget,
                                args.serve_max_particles, args.serve_target_ms, args.warmup)
    fifo = None if args.no_fifo else serve_one_at_a_time(apbf, torch, temps, descs, arrivals, args.serve_seconds)
    d.barrier()
    clock_info = clocks.stop()
    offered = sum(temps[k].n * steps for _, k, steps in arrivals) / args.serve_seconds
    value = d.sum(pooled["particle_steps_per_s"])
    ticks = pooled["ticks"]
    line = {
        "metric": SERVE_METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": d.ws,
        "steps": ticks, "warmup": args.warmup, "ms_per_step": pooled["step_ms_p50"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "apbf_serve", "arrivals_per_s": 200.0, "seconds": args.serve_seconds,
                   "particles_per_scene": "log-uniform 4096..262144 (64 seeded templates)",
                   "steps_per_scene": "uniform 30..300", "n_range": f"{c0.n_min}..{c0.n_max}",
                   "budget_gb": args.serve_budget_gb, "pool_gb": pooled["pool_gb"],
                   "capacity_particles": pooled["capacity_particles"], "capacity_cells": pooled["capacity_cells"],
                   "admission": "FIFO while particles, cells and scenes fit the pool",
                   "l2": "no flush: resident state far above 129 MB", "launch": "one captured graph per membership"},
        "offered_particle_steps_per_s": offered,
        "particle_iterations_per_s": d.sum(pooled["particle_iterations_per_s"]),
        "step_ms_p50": pooled["step_ms_p50"], "step_ms_p99": pooled["step_ms_p99"],
        "pooled": pooled, "latency_target": targeted, "one_at_a_time": fifo,
        "pooled_vs_one_at_a_time": ({"particle_steps": pooled["particle_steps_per_s"] / fifo["particle_steps_per_s"],
                                     "particle_iterations": pooled["particle_iterations_per_s"]
                                     / fifo["particle_iterations_per_s"]} if fifo else None),
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": pooled["h2d_bytes"] / max(1, ticks),
                "d2h_bytes_per_step": pooled["d2h_bytes"] / max(1, ticks),
                "what": "wall clock of the serving loop: host submit, admission uploads, ticks, result readback"},
        "roofline": None,
        "gpu_launches": ticks * kernels_per_step(c0),
        "clocks": clock_info,
    }
    if d.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serve_cpu_baseline(temps, rho0)
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


def serve_cpu_baseline(temps, rho0, budget_s=20.0):
    """The oracle on the host cores (OpenMP over particles): particle-steps/s
    over one step of each of the smallest serving templates until the budget
    is spent."""
    import oracle

    cores = oracle.set_threads(host_cores())
    t_used, n_used, done = 0.0, 0, 0
    for c in sorted(temps, key=lambda c: c.n):
        x, v = scenes.make_scene(c)
        p = oracle.make_params(c, rho0=rho0, eye=c.eye)
        t0 = time.perf_counter()
        oracle.step(p, x, v)
        t_used += time.perf_counter() - t0
        n_used += c.n
        done += 1
        if t_used > budget_s:
            break
    return {"value": n_used / t_used, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"one oracle step of each of the {done} smallest of {len(temps)} serving templates "
                      f"({n_used} particles)", "sample_seconds": t_used}


def batch_cpu_baseline(cfgs, rho0, budget_s=20.0):
    """The oracle on the host cores (OpenMP over particles), stepping the
    batch's scenes in order until the budget is spent; the per-particle time
    scaled to the whole batch."""
    import oracle

    cores = oracle.set_threads(host_cores())
    t_used, n_used, done = 0.0, 0, 0
    for c in sorted(cfgs, key=lambda c: c.n):
        x, v = scenes.make_scene(c)
        p = oracle.make_params(c, rho0=rho0, eye=c.eye)
        t0 = time.perf_counter()
        oracle.step(p, x, v)
        t_used += time.perf_counter() - t0
        n_used += c.n
        done += 1
        if t_used > budget_s:
            break
    n_total = sum(c.n for c in cfgs)
    scale = n_total / n_used
    return {"value": t_used * 1e3 * scale, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one oracle step of the {done} smallest of the {len(cfgs)} scenes ({n_used} of {n_total} "
                      f"particles), time x {scale:.3g}", "sample_seconds": t_used}


def run_lod_analysis(args, apbf, torch, d):
    """Where the adaptive models put the iterations: the workload stepped as
    APBF with the distance-to-camera model (DTC), APBF with the
    distance-to-the-visible-surface model (DTVS) and PBF with N_max, side by
    side on identical inputs and drivers; every `--analysis-every` steps,
    each run's particles per level N_i (from |P_l|), its mean N_i, its density
    error, and for DTVS the share of particles outside the view (they take
    N_min)."""
    cfg = workload(args.workload, "apbf")
    rho0 = float(np.float32(apbf.apbf_rest_density(cfg.h, cfg.mass, cfg.spacing)))
    runs = {"dtc": cfg, "dtvs": workload(args.workload, "dtvs"), "pbf_nmax": workload(args.workload, "pbf")}
    sc = {k: make_scene(apbf, c, rho0) for k, c in runs.items()}
    series = {k: [] for k in runs}
    for step in range(args.steps):
        for k, c in runs.items():
            drive(apbf, sc[k], c, step)
            apbf.apbf_step(sc[k], 1)
        if (step + 1) % args.analysis_every and step + 1 != args.steps:
            continue
        for k, c in runs.items():
            info = apbf.apbf_get_step_info(sc[k])
            ac = info["active_count"].astype(np.int64)
            per_level = {int(lv): int(ac[lv] - ac[lv + 1]) for lv in range(c.n_min, c.n_max + 1)
                         if ac[lv] - ac[lv + 1] > 0}
            row = {"step": step + 1, "mean_level": info["particle_iterations"] / c.n, "per_level": per_level,
                   "density": [float(v) for v in apbf.apbf_density_stats(sc[k])]}
            if k == "dtvs":
                dist = apbf.apbf_debug_read(sc[k], apbf.APBF_DBG_LOD_DISTANCE)
                row["outside_view"] = float(np.mean(dist < 0.0))
                row["visible"] = float(np.mean(dist == 0.0))
                row["d_range"] = [float(v) for v in info["d_range"]]
            series[k].append(row)
        print(f"step {step + 1}: " + "  ".join(f"{k} mean N {series[k][-1]['mean_level']:.2f} "
                                               f"|rho/rho0-1| {100 * series[k][-1]['density'][0]:.3f} %"
                                               for k in runs), file=sys.stderr, flush=True)
    line = {"metric": "LOD analysis: particles per level, mean N_i and density error of DTC, DTVS and PBF N_max",
            "value": None, "unit": None, "n_gpus": d.ws, "steps": args.steps, "warmup": 0, "dtype": "f32",
            "data": "synthetic", "config": workload_config(cfg, runs["pbf_nmax"].n_max, d.ws),
            "dtvs_view": {"width": DTVS_VIEW[0], "height": DTVS_VIEW[1], "fov_y_deg": 60.0,
                          "radius": 0.5 * cfg.spacing},
            "series": series}
    for k in sc:
        apbf.apbf_destroy_scene(sc[k])
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


def run_reference(args):
    """Reference arm: the CPU oracle, timed on the host cores, on this arm's
    workload; each step is a bounded sample (the bottom lattice layers of the
    same scene), the per-step time scaled by particles."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "batch_256":
        return run_reference_batch(args, ws)
    if args.workload == "serve":
        return run_reference_serve(args, ws)
    cfg = workload(args.workload, "apbf")
    pbf_cfg = workload(args.workload, "pbf")
    import oracle

    rho0 = float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))
    budget = float(os.environ.get("APBF_REFERENCE_BUDGET_S", "240"))
    cores = host_cores()
    # calibrate with one full step; the timed steps continue the trajectory from its state
    ms0, used, state = oracle_step_ms(oracle, cfg, rho0, 0, cores)
    full = (args.steps + args.warmup) * ms0 * 1e-3 <= budget
    sub, scale = cfg, 1.0
    if not full:
        # W + K whole steps would not fit the budget: the bottom lattice layers of the same scene
        nx, ny, nz = cfg.lattice
        layers = int(max(1, min(nz, nz * budget / ((args.steps + args.warmup) * ms0 * 1e-3))))
        sub = cfg.replace(lattice=(nx, ny, layers))
        scale = cfg.n / sub.n
        state = (None, None, None)
    x, v, ids = state
    times = []
    for s in range(args.warmup + args.steps):
        ms, _, (x, v, ids) = oracle_step_ms(oracle, sub, rho0, s + (1 if full else 0), cores, x, v, ids)
        if s >= args.warmup:
            times.append(ms * scale)
    value = float(np.mean(times))
    if full:
        sample = (f"each step: one oracle step of the whole workload ({cfg.n} particles, the trajectory's camera "
                  f"and wall), OpenMP over particles on {used} threads")
    else:
        sample = (f"each step: one oracle step of {sub.n} of the {cfg.n} particles (bottom {sub.lattice[2]} of "
                  f"{cfg.lattice[2]} lattice layers, same basin, camera, wall and N_i range) on {used} threads, "
                  f"time x {scale:g}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cfg, pbf_cfg.n_max, ws),
            "p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "nproc": cores,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_serve(args, ws):
    """Reference arm for the served workload: the oracle's particle-steps/s,
    each step one oracle step of the smallest serving templates that fit the
    per-step budget."""
    import oracle

    temps = sorted(scenes.config_serve_templates(), key=lambda c: c.n)
    c0 = temps[0]
    rho0 = float(np.float32(oracle.rest_density(c0.h, c0.mass, c0.spacing)))
    cores = oracle.set_threads(host_cores())
    budget = float(os.environ.get("APBF_REFERENCE_BUDGET_S", "150")) / max(1, args.steps + args.warmup)
    states, t_cal = [], 0.0
    for c in temps:
        x, v = scenes.make_scene(c)
        p = oracle.make_params(c, rho0=rho0, eye=c.eye)
        t0 = time.perf_counter()
        oracle.step(p, x, v)
        t_cal += time.perf_counter() - t0
        states.append([c, p, x, v, np.arange(c.n, dtype=np.int32)])
        if t_cal > budget:
            break
    n_used = sum(st[0].n for st in states)
    rates = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for st in states:
            out = oracle.step(st[1], st[2], st[3], st[4])
            st[2], st[3], st[4] = out.x, out.v, out.ids
        if s >= args.warmup:
            rates.append(n_used / (time.perf_counter() - t0))
    value = float(np.mean(rates))
    sample = f"each step: one oracle step of each of the {len(states)} smallest serving templates ({n_used} particles)"
    line = {"impl": "reference", "metric": SERVE_METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "apbf_serve", "n_range": f"{c0.n_min}..{c0.n_max}"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args, ws):
    """Reference arm for the batch: each step, the oracle steps the smallest
    scenes of the batch that fit the per-step budget, the time scaled by
    particles to the whole batch."""
    import oracle

    cfgs = sorted(scenes.config_batch_256(), key=lambda c: c.n)
    c0 = cfgs[0]
    rho0 = float(np.float32(oracle.rest_density(c0.h, c0.mass, c0.spacing)))
    cores = oracle.set_threads(host_cores())
    budget = float(os.environ.get("APBF_REFERENCE_BUDGET_S", "150")) / max(1, args.steps + args.warmup)
    states = []
    t_cal = 0.0
    for c in cfgs:   # calibrate: one step per scene until the per-step budget is reached
        x, v = scenes.make_scene(c)
        p = oracle.make_params(c, rho0=rho0, eye=c.eye)
        t0 = time.perf_counter()
        oracle.step(p, x, v)
        t_cal += time.perf_counter() - t0
        states.append([c, p, x, v, np.arange(c.n, dtype=np.int32)])
        if t_cal > budget:
            break
    n_total = sum(c.n for c in cfgs)
    n_used = sum(st[0].n for st in states)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for st in states:
            out = oracle.step(st[1], st[2], st[3], st[4])
            st[2], st[3], st[4] = out.x, out.v, out.ids
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt * 1e3 * n_total / n_used)
    value = float(np.mean(times))
    sample = (f"each step: one oracle step of each of the {len(states)} smallest of the {len(cfgs)} scenes "
              f"({n_used} of {n_total} particles), time x {n_total / n_used:.3g}")
    line = {"impl": "reference", "metric": "batched APBF ms/step for 256 independent scenes vs one at a time",
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "apbf_batch_256", "scenes": len(cfgs), "particles": n_total,
                       "n_range": f"{c0.n_min}..{c0.n_max}", "lod": "distance to camera"},
            "p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def default_steps(name: str) -> int:
    """A workload's own length in steps (the batch: its scenes' 100 steps)."""
    if name in ("batch_256", "serve"):
        return 100
    return int(workload(name, "apbf").steps)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's own length: 600 for the ocean, 300 for the 131k and "
                         "225k scenes, 20 for the 4k dam break, 100 for the batch)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ocean_1m",
                    choices=["ocean_1m", "dam_break_131k", "multi_dam_break_225k", "dam_break_4k", "batch_256",
                             "serve"])
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-max-particles", type=int, default=0)
    ap.add_argument("--serve-target-ms", type=float, default=33.3,
                    help="step-latency target of the second pooled run (0: skip that run)")
    ap.add_argument("--no-fifo", action="store_true", help="skip the one-scene-at-a-time serving arm")
    ap.add_argument("--lod-analysis", action="store_true",
                    help="record particles per level and density of DTC, DTVS and PBF N_max instead of timing")
    ap.add_argument("--analysis-every", type=int, default=50)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-pbf", action="store_true")
    ap.add_argument("--no-dtvs", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = default_steps(args.workload)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_1608_04721_gb300 import apbf, build

    d = Dist()
    torch.cuda.set_device(d.local)
    build.build()
    apbf.lib()
    if args.workload == "batch_256":
        return run_batch(args, apbf, torch, d)
    if args.workload == "serve":
        return run_serve(args, apbf, torch, d)
    if args.lod_analysis:
        return run_lod_analysis(args, apbf, torch, d)
    cfg = workload(args.workload, "apbf")
    pbf_cfg = workload(args.workload, "pbf")
    rho0 = float(np.float32(apbf.apbf_rest_density(cfg.h, cfg.mass, cfg.spacing)))

    dtvs_cfg = workload(args.workload, "dtvs")
    flush = needs_flush(cfg.n)
    scene = make_scene(apbf, cfg, rho0)
    pbf = None if args.no_pbf else make_scene(apbf, pbf_cfg, rho0)
    pbf_lo_cfg = workload(args.workload, "pbf_nmin")
    pbf_lo = None if args.no_pbf else make_scene(apbf, pbf_lo_cfg, rho0)
    dtvs = None if args.no_dtvs else make_scene(apbf, dtvs_cfg, rho0)
    tuning = {}
    if not args.no_autotune:
        # trial steps run on a snapshot that the tuner restores, so the timed trajectory is unchanged
        drive(apbf, scene, cfg, 0)
        tuning["apbf"] = tune_summary(apbf.apbf_autotune(scene, 4))
        if pbf is not None:
            drive(apbf, pbf, pbf_cfg, 0)
            tuning["pbf_nmax"] = tune_summary(apbf.apbf_autotune(pbf, 4))
            drive(apbf, pbf_lo, pbf_lo_cfg, 0)
            tuning["pbf_nmin"] = tune_summary(apbf.apbf_autotune(pbf_lo, 4))
        if dtvs is not None:
            drive(apbf, dtvs, dtvs_cfg, 0)
            tuning["apbf_dtvs"] = tune_summary(apbf.apbf_autotune(dtvs, 4))
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    # ---- APBF, device-resident inputs
    d.barrier()
    torch.cuda.synchronize()
    tot, per, s_next = timed_run(apbf, torch, scene, cfg, args.warmup, args.steps, flush=flush)
    torch.cuda.synchronize()
    d.barrier()
    ms_step = d.max(tot / args.steps)
    apbf_density = apbf.apbf_density_stats(scene)
    # ---- PBF(N_min) on identical inputs and drivers: the other end of the adaptive range
    pbf_lo_line = None
    if pbf_lo is not None:
        d.barrier()
        ltot, lper, _ = timed_run(apbf, torch, pbf_lo, pbf_lo_cfg, args.warmup, args.steps, flush=flush)
        d.barrier()
        pbf_lo_line = {"ms_per_step": d.max(ltot / args.steps), "p50_ms": metrics.percentile(lper, 50),
                       "p99_ms": metrics.percentile(lper, 99), "n": pbf_lo_cfg.n_max,
                       "density": [float(v) for v in apbf.apbf_density_stats(pbf_lo)]}
    # ---- PBF(N_max) on identical inputs and drivers
    pbf_line = None
    if pbf is not None:
        d.barrier()
        ptot, pper, _ = timed_run(apbf, torch, pbf, pbf_cfg, args.warmup, args.steps, flush=flush)
        d.barrier()
        pbf_ms = d.max(ptot / args.steps)
        pbf_density = apbf.apbf_density_stats(pbf)
        pbf_line = {"ms_per_step": pbf_ms, "p50_ms": metrics.percentile(pper, 50),
                    "p99_ms": metrics.percentile(pper, 99), "n": pbf_cfg.n_max,
                    "density": [float(v) for v in pbf_density]}
    # ---- APBF with the DTVS model on identical inputs and drivers
    dtvs_line = None
    if dtvs is not None:
        d.barrier()
        dtot, dper, ds_next = timed_run(apbf, torch, dtvs, dtvs_cfg, args.warmup, args.steps, flush=flush)
        d.barrier()
        dtvs_ms = d.max(dtot / args.steps)
        dtvs_density = apbf.apbf_density_stats(dtvs)
        dms, _, _, _, diters, _ = stage_profile(apbf, dtvs, dtvs_cfg, ds_next, min(args.profile_steps, 20))
        nprof = min(args.profile_steps, 20)
        dtvs_line = {"ms_per_step": dtvs_ms, "p50_ms": metrics.percentile(dper, 50),
                     "p99_ms": metrics.percentile(dper, 99),
                     "view": {"width": DTVS_VIEW[0], "height": DTVS_VIEW[1], "fov_y_deg": 60.0,
                              "radius": 0.5 * dtvs_cfg.spacing},
                     "lod_stage_ms": float(dms[0] / nprof),
                     "particle_iterations_per_step": diters / nprof,
                     "density": [float(v) for v in dtvs_density]}
        # the same with the particles outside the view at n_max instead of n_min
        # (apbf_set_view_outside_level), on identical inputs and drivers
        dtvs_hi = make_scene(apbf, dtvs_cfg, rho0)
        apbf.apbf_set_view_outside_level(dtvs_hi, dtvs_cfg.n_max)
        if "apbf_dtvs" in tuning:
            apbf.apbf_set_tuning(dtvs_hi, tuning["apbf_dtvs"]["block"], tuning["apbf_dtvs"]["mask_threshold"])
        d.barrier()
        htot, hper, hs_next = timed_run(apbf, torch, dtvs_hi, dtvs_cfg, args.warmup, args.steps, flush=flush)
        d.barrier()
        hdens = apbf.apbf_density_stats(dtvs_hi)
        _, _, _, _, hiters, _ = stage_profile(apbf, dtvs_hi, dtvs_cfg, hs_next, 5)
        dtvs_line["outside_nmax"] = {"ms_per_step": d.max(htot / args.steps), "p50_ms": metrics.percentile(hper, 50),
                                     "p99_ms": metrics.percentile(hper, 99),
                                     "particle_iterations_per_step": hiters / 5,
                                     "density": [float(v) for v in hdens]}
        apbf.apbf_destroy_scene(dtvs_hi)
    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_scene = make_scene(apbf, cfg, rho0)
        if "apbf" in tuning:
            apbf.apbf_set_tuning(e2e_scene, tuning["apbf"]["block"], tuning["apbf"]["mask_threshold"])
        host_pos = torch.empty((cfg.n, 3), dtype=torch.float32, pin_memory=True).numpy()
        bufs = [torch.empty((cfg.n, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        for k in range(args.warmup):
            drive(apbf, e2e_scene, cfg, k)
            apbf.apbf_step(e2e_scene, 1)
            apbf.apbf_read_state(e2e_scene, pos=host_pos, vel=False)
        # pipelined, as a renderer consumes it: step k's positions are copied
        # into one of two pinned buffers while step k + 1 computes
        d.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            drive(apbf, e2e_scene, cfg, args.warmup + k)   # camera + wall: host -> device
            apbf.apbf_step(e2e_scene, 1)
            apbf.apbf_read_positions_async(e2e_scene, bufs[k % 2].data_ptr())  # positions: device -> host
        apbf.apbf_sync(e2e_scene)
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        # synchronous: each step's positions are on the host before the next step is queued
        k0 = args.warmup + args.steps
        d.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            drive(apbf, e2e_scene, cfg, k0 + k)
            apbf.apbf_step(e2e_scene, 1)
            apbf.apbf_read_state(e2e_scene, pos=host_pos, vel=False)
        sync_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        d.barrier()
        e2e_ms, sync_ms = d.max(e2e_ms), d.max(sync_ms)
        e2e = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 64, "d2h_bytes_per_step": 12 * cfg.n,
               "what": "per step: apbf_set_camera + apbf_set_box (64 B upload), apbf_step, "
                       "apbf_read_positions_async of all positions into one of two pinned host buffers (the copy "
                       "overlaps the next step), apbf_sync after the last step; host wall clock",
               "sync_value": sync_ms,
               "sync_what": "the same with apbf_read_state (synchronising) every step"}
        apbf.apbf_destroy_scene(e2e_scene)
    clock_info = clocks.stop()

    # ---- per-stage device times (eager launches with events) for the roofline
    ms_st, ln_st, pairs, nbr_pairs, iters, _ = stage_profile(apbf, scene, cfg, s_next, args.profile_steps)
    stage_ms = {STAGE_NAMES[k]: float(ms_st[k] / args.profile_steps) for k in range(len(STAGE_NAMES))}
    top = max(("lambda", "deltap"), key=lambda k: stage_ms[k])
    k_top = STAGE_NAMES.index(top)
    launches = max(1.0, float(ln_st[k_top]))
    avg_launch_s = ms_st[k_top] / launches * 1e-3
    flops_per_launch = FLOPS_PER_PAIR[top] * pairs / launches
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops_per_launch / avg_launch_s / 1e12
    traffic = read_traffic(f"{top}_kernel", cfg.name)
    roofline = {"bound": "alu", "kernel": f"{top}_kernel", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz",
                "limiter": LIMITER_NOTE,
                "flops_per_pair": FLOPS_PER_PAIR[top], "pairs_per_launch": pairs / launches,
                "avg_launch_us": avg_launch_s * 1e6}
    particle_iters_per_step = iters / args.profile_steps
    dims = apbf.apbf_debug_dims(scene)[0]
    stage_hbm = stage_roofline(stage_ms, cfg.n, int(dims[0]) * int(dims[1]) * int(dims[2]), torch, level_entries(cfg))
    value = ms_step
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(cfg, pbf_cfg.n_max, d.ws),
        "launch": "captured CUDA graph per step",
        "tuning": tuning or "defaults (block 256, compacted levels)",
        "p50_ms": metrics.percentile(per, 50), "p99_ms": metrics.percentile(per, 99),
        "particle_iterations_per_step": particle_iters_per_step,
        "particle_iterations_per_s": d.sum(particle_iters_per_step / (ms_step * 1e-3)),
        "neighbor_pairs_per_step": nbr_pairs / args.profile_steps,
        "density": {"apbf": [float(v) for v in apbf_density],
                    "fields": ["mean|rho/rho0-1|", "max|rho/rho0-1|", "mean(rho/rho0-1)", "mean max(0,rho/rho0-1)"]},
        "pbf_nmax": pbf_line,
        "pbf_nmin": pbf_lo_line,
        "improvement": metrics.improvement(pbf_line["ms_per_step"], ms_step) if pbf_line else None,
        "apbf_dtvs": dtvs_line,
        "improvement_dtvs": (metrics.improvement(pbf_line["ms_per_step"], dtvs_line["ms_per_step"])
                             if pbf_line and dtvs_line else None),
        "roofline": roofline,
        "stage_ms_per_step": stage_ms,
        "stage_roofline": stage_hbm,
        "e2e": e2e,
        "gpu_launches": kernels_per_step(cfg) * args.steps,
        "clocks": clock_info,
    }
    if pbf_line:
        line["density"]["pbf_nmax"] = pbf_line["density"]
        line["density"]["pbf_nmin"] = pbf_lo_line["density"]
        line["density"]["mean_abs_diff_points"] = 100 * abs(apbf_density[0] - pbf_line["density"][0])
    if d.rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    apbf.apbf_destroy_scene(scene)
    if pbf is not None:
        apbf.apbf_destroy_scene(pbf)
        apbf.apbf_destroy_scene(pbf_lo)
    if dtvs is not None:
        apbf.apbf_destroy_scene(dtvs)
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

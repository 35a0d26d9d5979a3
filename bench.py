"""Benchmark of the per-frame particle update (gradient-guided Monte Carlo SLAM).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

One step = one frame of the whole hot path on the paper-scale session:
100,000 particles, 2,048-point scans, 20 keyframes of 8,192 points (0.2 m
lattice), 3 neighbour keyframes, 3 gradient-guided moves, the value pass,
log-sum-exp weighting and systematic resampling. Inputs are synthetic (a
procedural corridor-and-trunk scene ray-cast by a 64 x 1024 lidar), resident
in HBM before the timed region. L2 is flushed (a 256 MB write) before every
timed step, outside its events.

Metric: particle x point likelihood+gradient evaluations per second, i.e.
P * N * steps per frame (each evaluation covers the 3 neighbour keyframes);
the frame time p50/p99 and lookups/s are reported beside it.

Under torchrun (N > 1) every rank runs an independent session (replicas: the
filter has no data-path exchange); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle×point lik+grad evals/s; frame update ms @100k particles; p50/p99"
UNIT = "evals/s"
# FP32 flops of one gradient lookup of a move (FMA = 2): transform 18, floor and
# fraction 6, value from the trilinear coefficients 14 and its gradient 8, L + eps and
# the reciprocal 2, normalised gradient and weight 4, accumulation 16, moments 19 per
# point shared by its 3 lookups; the moves do not need the log-likelihood. Every
# table type stores coefficients (16-bit records are widened, which is no flop).
FLOPS_GRAD_LOOKUP = {"f32": 74, "bf16": 74, "f16": 74}
# GICP model: FP32 flops (FMA = 2) of an inlier lookup with the Gauss-Newton terms in
# the keyframe-frame form the kernel uses, and of a lookup that stops at an empty voxel
# (transform and cell only); lookups rejected by the cap are counted as the latter
FLOPS_GICP_INLIER = 198
FLOPS_GICP_MISS = 24
GICP_VOXEL = 1.0                # m, voxel edge of the GICP keyframe maps
FP32_LANES_PER_SM = 128         # FP32 FMA lanes per SM (4 schedulers x 32)
# DRAM bytes read + written per gradient-pass launch, from one ncu capture of the
# current kernel on dense tables at 100,000 particles x 2,048 points (profiles/);
# reported only for that workload (elsewhere the tables' share of L2 differs, so the
# traffic does not scale with the lookups)
TRAFFIC_PER_LAUNCH = {"f32": 32.59e6, "bf16": 30.52e6, "f16": 30.51e6}
TRAFFIC_WORKLOAD = (100_000, 2048, "dense")


def max_sm_mhz(index):
    """Maximum SM clock of GPU `index` (nvidia-smi), else the driver-measured
    MEASURED_PEAKS.json figure, else the part's nominal 2032 MHz."""
    try:
        out = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        return float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
    except Exception:
        pass
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]), "MEASURED_PEAKS.json"
    except Exception:
        return 2032.0, "nominal"


def fp32_peak(dev_index, g):
    """FP32 peak from the unit counts: the SM count read from the device x 128
    lanes x 2 flop x the maximum SM clock; beside it the measured FMA rate."""
    ffma, sms = g.probe_ffma()
    mhz, src = max_sm_mhz(dev_index)
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, (f"{sms} SMs (read from the device) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:.0f} MHz "
                  f"({src}); measured FFMA rate {ffma:.1f} TFLOP/s (gmcs_probe_ffma)"), ffma, sms


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--particles", type=int, default=100_000)
    ap.add_argument("--points", type=int, default=2048)
    ap.add_argument("--keyframes", type=int, default=20)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--layout", default="dense", choices=["dense", "columns"],
                    help="likelihood tables: dense lattices, or column-sparse (only each (x, y) column's run of "
                         "nonzero cells)")
    ap.add_argument("--model", default="field", choices=["field", "gicp"],
                    help="likelihood: voxel field (the benchmark's) or GICP distribution-to-distribution (Eq. 2-6)")
    ap.add_argument("--resample", default="always", choices=["always", "ess", "never", "prune"],
                    help="resampling policy (always: the benchmark's systematic resampling every frame; "
                         "prune: the paper's dead-particle pruning)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-particles", type=int, default=8192,
                    help="oracle sample for cpu_baseline, split over the host cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    ap.add_argument("--serve", action="store_true", help="serving benchmark (32 sessions, continuous batching)")
    ap.add_argument("--sessions", type=int, default=32)
    ap.add_argument("--session-frames", type=int, default=20)
    ap.add_argument("--budget-gb", type=float, default=80.0)
    ap.add_argument("--serve-range", type=float, default=20.0, help="lidar range of the serving scenes (m)")
    ap.add_argument("--serve-pool", type=int, default=60, help="distinct keyframe clouds shared by the sessions")
    ap.add_argument("--serve-rate", type=float, default=10.0, help="frames per second per session")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-at-a-time plain FP32 comparison")
    ap.add_argument("--serve-dtype", default="bf16", choices=["f32", "bf16", "f16"],
                    help="table storage of the served sessions")
    ap.add_argument("--tick-work", type=float, default=None,
                    help="server cap on the evals a tick gathers (default: the library's; 0 lifts it)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed plumbing
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist


def reduce_max(value, world, device=None):
    """Max of a float over ranks (identity at world size 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world, device=None):
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock, max clock and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
def oracle_prepare(w, n_particles, model="field"):
    """FP64 oracle state for the first n_particles of the workload, with tables
    (GICP: voxel maps) for every keyframe a sampled particle can select (an
    empty 2x2x2 lattice far away, which every lookup misses, stands in for the
    others)."""
    import oracle
    import synth
    P = n_particles
    K = len(w["keyframes"])
    poses = w["particles"][:P].astype(np.float64)
    kfp = np.stack([p[:P] for p in w["kf_particle_poses"]]).astype(np.float64)
    t = poses[:, [3, 7, 11]]
    dist = np.stack([np.linalg.norm(kfp[k][:, [3, 7, 11]] - t, axis=1) for k in range(K)], 1)
    third = np.sort(dist, axis=1)[:, min(2, K - 1)]
    need = set(np.nonzero((dist <= third[:, None] + 3.0).any(axis=0))[0].tolist())
    tables, grids = [], []
    for k, kf in enumerate(w["keyframes"]):
        if k in need and model == "gicp":
            grid = synth.grid_for_points(kf["points"], GICP_VOXEL, 1.0)
            tables.append(oracle.gicp_voxel_map(kf["points"], oracle.knn_cov(kf["points"], 10), grid))
            grids.append(grid)
        elif k in need:
            tables.append(oracle.build_table(kf["points"], kf["grid"], 0.2, 1.0))
            grids.append(kf["grid"])
        else:
            tables.append(np.zeros((1, 10)) if model == "gicp" else np.zeros((2, 2, 2)))
            grids.append({"origin": np.array([1e6, 1e6, 1e6]), "h": 1.0,
                          "dims": (1, 1, 1) if model == "gicp" else (2, 2, 2)})
    return oracle.State(poses, kfp, tables, grids)


POLICY = {"always": 0, "ess": 1, "never": 2, "prune": 3}


def oracle_frames(st, w, frames, first=0, model="field", resample="always"):
    """Seconds of each whole oracle frame (single thread) on the prepared sample
    (GICP: the scan covariances are part of the frame)."""
    import oracle
    out = []
    for fr in range(first, first + frames):
        t0 = time.perf_counter()
        if model == "gicp":
            st.step(w["scans"][fr], w["odometry"][fr], w["cov"], frame=fr, scov=oracle.knn_cov(w["scans"][fr], 10),
                    model=1, resample=POLICY[resample])
        else:
            st.step(w["scans"][fr], w["odometry"][fr], w["cov"], frame=fr, resample=POLICY[resample])
        out.append(time.perf_counter() - t0)
    return np.array(out)


# Per-worker oracle states and the workload, set in the parent before the pool
# forks; the forked workers read them (copy-on-write), so nothing large is pickled.
_POOL_STATES = None
_POOL_W = None


def _pool_frame(task):
    i, fr, model, resample = task
    return float(oracle_frames(_POOL_STATES[i], _POOL_W, 1, first=fr, model=model, resample=resample)[0])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle on the host cores: one forked worker per core, each running
    whole oracle frames on its own block of the session's particles (the tables
    are built once in the parent and shared). Must be created before the process
    first touches CUDA: a pool forked after that can hang."""

    def __init__(self, w, total_particles, model="field", max_workers=64, resample="always"):
        import multiprocessing as mp
        import oracle
        global _POOL_STATES, _POOL_W
        self.workers = max(1, min(host_cores(), max_workers))
        self.per_worker = max(16, total_particles // self.workers)
        self.model = model
        self.resample = resample
        n = min(self.per_worker * self.workers, w["particles"].shape[0])
        self.per_worker = n // self.workers
        base = oracle_prepare(w, self.per_worker * self.workers, model)
        b = self.per_worker
        _POOL_STATES = [oracle.State(base.poses[i * b:(i + 1) * b], base.kf_poses[:, i * b:(i + 1) * b],
                                     base.tables, base.grids) for i in range(self.workers)]
        _POOL_W = w
        self.pool = mp.get_context("fork").Pool(self.workers)

    def frame(self, fr):
        """Wall seconds of frame fr on every worker's block at once, and the
        workers' own seconds."""
        t0 = time.perf_counter()
        per = self.pool.map(_pool_frame, [(i, fr, self.model, self.resample) for i in range(self.workers)],
                            chunksize=1)
        return time.perf_counter() - t0, per

    def close(self):
        self.pool.close()
        self.pool.join()


# ----------------------------------------------------------------------------- native arm
def run_native(a, world, rank, local):
    import torch
    import paper_2504_18056_b300 as g
    import synth

    frames = a.warmup + a.steps + a.e2e_steps
    w = synth.forest_workload(seed=rank, n_particles=a.particles, n_points=a.points, n_keyframes=a.keyframes,
                              n_frames=frames)
    # the oracle's worker pool forks before this process touches CUDA
    opool = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        opool = OraclePool(w, a.cpu_particles if a.model != "gicp" else a.cpu_particles // 4, model=a.model,
                           resample=a.resample)
    torch.cuda.set_device(local)
    torch.cuda.init()
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    P, N, K = a.particles, a.points, a.keyframes
    dtype = {"f32": 0, "bf16": 1, "f16": 2}[a.dtype]
    gicp = a.model == "gicp"
    stream = torch.cuda.current_stream(dev)
    layout = g.LAYOUT_COLUMNS if a.layout == "columns" else g.LAYOUT_DENSE
    f = g.Filter(P, K, N, stream=stream.cuda_stream, table_dtype=dtype, seed=rank,
                 model=g.MODEL_GICP if gicp else g.MODEL_FIELD, resample=POLICY[a.resample], table_layout=layout)
    f.init_particles(w["particles"])
    for k, kf in enumerate(w["keyframes"]):
        grid = synth.grid_for_points(kf["points"], GICP_VOXEL, 1.0) if gicp else kf["grid"]
        f.add_keyframe(kf["points"], grid, w["kf_particle_poses"][k])
    scans_d = [torch.from_numpy(s).to(dev) for s in w["scans"]]
    flush = None if a.no_flush else torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    torch.cuda.synchronize()

    for fr in range(a.warmup):
        f.step(scans_d[fr], w["odometry"][fr], w["cov"], sync=False)
    torch.cuda.synchronize()

    # L2 gather ceiling: random cell-record reads from a 64 MB buffer (fits the 126 MB L2)
    l2_gbs = None if gicp else g.probe_gather(64 << 20, 32 if dtype == 0 else 16)
    peak_tflops, peak_src_fp32, ffma_tflops, sm_count = fp32_peak(local, g)
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    f.set_profiling(True)
    f.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for s in range(a.steps):
        fr = a.warmup + s
        if not a.no_flush:
            flush.fill_(float(s))
        ev[s][0].record(stream)
        f.step(scans_d[fr], w["odometry"][fr], w["cov"], sync=False)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    stats = f.stats()
    f.set_profiling(False)
    res = f.last_result()

    # end to end through the public call: pinned host scan in, result struct out
    pinned = [torch.from_numpy(w["scans"][a.warmup + a.steps + s]).pin_memory() for s in range(a.e2e_steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(a.e2e_steps):
        fr = a.warmup + a.steps + s
        out = f.step(pinned[s], w["odometry"][fr], w["cov"])      # synchronises, fills the host struct
    e2e_s = time.perf_counter() - t0
    assert out["status"] == 0
    dev_bytes = f.device_bytes()
    inlier_frac = None
    if gicp:
        # share of lookups that reach a distribution and pass the cap, at the final state
        mom = torch.zeros((P, 22), dtype=torch.float32, device=dev)
        f.eval(scans_d[a.warmup + a.steps - 1], None, None, mom)
        inlier_frac = float(mom[:, 21].sum().item()) / (float(P) * N * 3)
    f.close()

    total_ms = float(step_ms.sum())
    max_ms = reduce_max(total_ms, world, dev)
    evals_rank = float(P) * N * 3 * a.steps
    evals_all = reduce_sum(evals_rank, world, dev)
    value = evals_all / (max_ms / 1e3)
    e2e_max = reduce_max(e2e_s, world, dev)
    e2e_value = reduce_sum(float(P) * N * 3 * a.e2e_steps, world, dev) / e2e_max

    kinds = stats["kinds"]
    pg = kinds["pass_grad"]
    lookups_per_launch = float(P) * N * 3
    rec_bytes = 32 if dtype == 0 else 16
    avg_ms = pg["ms"] / max(pg["launches"], 1)
    # algorithmic work of one gradient lookup: 74 FP32 flops (FMA = 2), one cell record read;
    # GICP: 198 per inlier, 24 per other lookup, 48 B voxel record per lookup
    if gicp:
        flops_per_launch = lookups_per_launch * (inlier_frac * FLOPS_GICP_INLIER + (1 - inlier_frac) * FLOPS_GICP_MISS)
        rec_bytes = 48
    else:
        flops_per_launch = lookups_per_launch * FLOPS_GRAD_LOOKUP[a.dtype]
    achieved_tflops = flops_per_launch / (avg_ms / 1e3) / 1e12
    gather_gbs = lookups_per_launch * rec_bytes / (avg_ms / 1e3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak, peak_src = 6400.0, "fallback"
    if os.path.exists(peaks_path):
        hbm_peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    timed_kernel_ms = sum(v["ms"] for v in kinds.values())
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": max_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16 tables, f32 math", "f16": "f16 tables, f32 math"}[a.dtype] +
                 "; f64 weights",
        "data": "synthetic (seeded procedural corridor + trunk scene, 64x1024 lidar ray-cast)",
        "config": {"workload": f"single session, {P} particles x {N}-point scans x {K} keyframes "
                               + ("(8192 pts, GICP voxel maps at 1 m, knn 10)" if gicp else "(8192 pts, 0.2 m lattice)")
                               + ", 3 neighbour keyframes, 3 moves/frame"
                               + (", column-sparse tables" if a.layout == "columns" else "")
                               + ("" if a.resample == "always" else f", resampling policy {a.resample}"),
                   "model": a.model, "resample": a.resample,
                   "particles": P, "points": N, "keyframes": K, "k_nb": 3, "moves": 3,
                   "table": a.dtype, "layout": a.layout,
                   "l2": "flushed before every timed step (256 MB write)" if not a.no_flush
                   else "not flushed", "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "frame_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                     "min": float(step_ms.min()), "max": float(step_ms.max())},
        "lookups_per_s": float(P) * N * 3 * 4 * a.steps * world / (max_ms / 1e3),
        "kernels_ms_per_step": {k: v["ms"] / a.steps for k, v in kinds.items() if v["launches"]},
        "roofline": {"kernel": "k_gicp gradient pass (GICP terms + Gauss-Newton matrix)" if gicp else
                               "k_pass3 gradient pass (lookup + gradient + moments)", "bound": "alu",
                     "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak_tflops,
                     "frac_of_measured_ffma": achieved_tflops / ffma_tflops, "measured_ffma_tflops": ffma_tflops,
                     "sm_count": sm_count,
                     "traffic": None if gicp or (a.particles, a.points, a.layout) != TRAFFIC_WORKLOAD
                     else TRAFFIC_PER_LAUNCH.get(a.dtype), "gicp_inlier_frac": inlier_frac,
                     "peak_source": peak_src_fp32,
                     "algorithmic_flops_per_launch": flops_per_launch, "avg_launch_ms": avg_ms},
        "gather": {"algorithmic_bytes_per_launch": lookups_per_launch * rec_bytes, "achieved_gbs": gather_gbs,
                   "hbm_peak_gbs": hbm_peak, "hbm_peak_source": peak_src, "frac_of_hbm": gather_gbs / hbm_peak,
                   "l2_gather_gbs": l2_gbs, "l2_gather_source": "gmcs_probe_gather, 64 MB buffer, random records",
                   "frac_of_l2_gather": gather_gbs / l2_gbs if l2_gbs else None,
                   "frame_at_hbm_roofline_ms": float(P) * N * 3 * 4 * rec_bytes / (hbm_peak * 1e9) * 1e3},
        "clocks": clk,
        "gpu_launches": int(stats["launches"]),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * 12,
                "d2h_bytes_per_step": 128, "frame_ms": e2e_max / a.e2e_steps * 1e3},
        "estimate_error_m": float(np.linalg.norm(res["estimate"][[3, 7, 11]] -
                                                 w["truth"][a.warmup + a.steps][[3, 7, 11]])),
        "device_bytes": dev_bytes,
        "timed_kernel_share": timed_kernel_ms / total_ms if total_ms > 0 else None,
    }
    if opool is not None:
        wall, per = opool.frame(0)
        opool.close()
        n_all = opool.per_worker * opool.workers
        desc = (f"FP64 oracle ({a.model} model), whole frame 0 of the same session on {n_all} of its particles: "
                f"{opool.workers} forked workers (one per host core) with {opool.per_worker} particles each, "
                f"{N} points, {K} keyframes, 3 moves")
        line["cpu_baseline"] = {"value": n_all * N * 3 / wall, "unit": UNIT, "cores": opool.workers,
                                "kind": "oracle", "sample": desc, "seconds": wall,
                                "cpu_seconds": float(np.sum(per)),
                                "per_core_value": opool.per_worker * N * 3 / float(np.median(per))}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return line


# ----------------------------------------------------------------------------- serving arm
def _setup_session(f, pool, spec, dev):
    """Particles from the host; keyframe clouds and per-particle keyframe poses
    from device buffers (no host round trip per keyframe)."""
    import torch
    f.init_particles(synth_session_particles(pool, spec))
    npool = len(pool["keyframes"])
    kf_buf = torch.empty((spec["P"], 12), dtype=torch.float32, device="cuda")
    for k in range(spec["K"]):
        kf = pool["keyframes"][k % npool]
        kf_buf.copy_(dev["kf_pose"][k % npool].expand(spec["P"], 12))
        torch.cuda.current_stream().synchronize()
        f.add_keyframe(dev["points"][k % npool], kf["grid"], kf_buf)


def synth_session_particles(pool, spec):
    import synth
    return synth.session_particles(pool, spec)


def _saturate(srv, sat_sids, a, pool, frame_idx):
    for i in range(a.session_frames):
        for sid, spec in sat_sids:
            fi = frame_idx(spec, i)
            srv.submit(sid, pool["scans"][fi][:spec["N"]], pool["odometry"][fi], pool["cov"])
    srv.drain()
    return srv.stats()


def run_serve(a):
    """Config 5: sessions with P ~ U[4096, 200000], N ~ U[1024, 8192], K ~ U[10, 300],
    Poisson frames at 10 Hz per session, admission by a device-memory budget;
    BF16 tables (or --serve-dtype) through the server, against the plain FP32 path
    serving the same sessions one at a time."""
    import torch
    import paper_2504_18056_b300 as g
    import synth

    torch.cuda.init()
    t0 = time.perf_counter()
    pool = synth.serving_pool(seed=0, n_kf=a.serve_pool, rmax=a.serve_range)
    specs = synth.serving_sessions(seed=0, n_sessions=a.sessions, n_frames=a.session_frames)
    t_gen = time.perf_counter() - t0
    nscan = len(pool["scans"])
    frame_idx = lambda spec, i: (spec["frame0"] + i) % nscan
    dev = {"points": [torch.from_numpy(kf["points"]).cuda() for kf in pool["keyframes"]],
           "kf_pose": [torch.from_numpy(kf["pose"].astype(np.float32)).cuda() for kf in pool["keyframes"]]}
    if a.serve_rate != 10.0:
        for sp in specs:
            sp["arrivals"] = sp["arrivals"] * (10.0 / a.serve_rate)

    sdt = {"f32": 0, "bf16": 1, "f16": 2}[a.serve_dtype]
    rec = 32 if sdt == 0 else 16        # bytes per cell record
    slayout = g.LAYOUT_COLUMNS if a.layout == "columns" else g.LAYOUT_DENSE
    # admission estimate of a keyframe's table: the dense lattice, or for column-sparse
    # tables a fifth of it (the server charges the actual bytes once the session is set up)
    table_share = 0.2 if a.layout == "columns" else 1.0
    srv = g.Server(budget_bytes=int(a.budget_gb * (1 << 30)), max_sessions=a.sessions, background=True,
                   table_dtype=sdt, table_layout=slayout)
    if a.tick_work is not None:
        srv.set_tick_work(a.tick_work)
    lat_by_work = []                    # (P x N of the session, server latency of one frame)
    waiting = list(range(len(specs)))
    active = {}
    e2e_lat = []
    done_sessions = 0
    setup_s = 0.0
    t_start = time.perf_counter()
    while done_sessions < len(specs):
        # admission: open sessions while the budget allows
        while waiting:
            spec = specs[waiting[0]]
            P, K, N = spec["P"], spec["K"], spec["N"]
            tb = int(K * (pool["keyframes"][0]["grid"]["dims"][0] * pool["keyframes"][0]["grid"]["dims"][1] *
                          pool["keyframes"][0]["grid"]["dims"][2]) * rec * table_share)
            sid = srv.open(P, K, N, table_bytes=tb, seed=spec["seed"])
            if sid is None:
                break
            ts = time.perf_counter()
            f = srv.session(sid)
            _setup_session(f, pool, spec, dev)
            srv.ready(sid)
            setup_s += time.perf_counter() - ts
            active[sid] = {"spec": spec, "t0": time.perf_counter(), "next": 0, "tickets": [], "done": 0, "late": []}
            waiting.pop(0)
        now = time.perf_counter()
        for sid, st in list(active.items()):
            spec = st["spec"]
            while st["next"] < len(spec["arrivals"]) and st["t0"] + spec["arrivals"][st["next"]] <= now:
                fi = frame_idx(spec, st["next"])
                t_sched = st["t0"] + spec["arrivals"][st["next"]]
                st["tickets"].append(srv.submit(sid, pool["scans"][fi][:spec["N"]], pool["odometry"][fi], pool["cov"]))
                st["late"].append(time.perf_counter() - t_sched)   # the request loop's own delay
                st["next"] += 1
            while st["done"] < len(st["tickets"]):
                r = srv.poll(st["tickets"][st["done"]])
                if r is None:
                    break
                e2e_lat.append(st["late"][st["done"]] + r[1])
                lat_by_work.append((spec["P"] * spec["N"], r[1]))
                st["done"] += 1
            if st["done"] == len(spec["arrivals"]):
                srv.close_session(sid)
                del active[sid]
                done_sessions += 1
        time.sleep(0.0005)
    wall = time.perf_counter() - t_start
    stats = srv.stats()

    # saturation: the sessions that fit the budget at once, every frame submitted together
    srv.reset_stats()
    sat_sids = []
    for spec in specs:
        tb = int(spec["K"] * int(np.prod(pool["keyframes"][0]["grid"]["dims"])) * rec * table_share)
        sid = srv.open(spec["P"], spec["K"], spec["N"], table_bytes=tb, seed=spec["seed"])
        if sid is None:
            break
        _setup_session(srv.session(sid), pool, spec, dev)
        srv.ready(sid)
        sat_sids.append((sid, spec))
    sat = {}
    for inflight in (2, 1):
        srv.set_inflight(inflight)
        srv.reset_stats()
        sat[inflight] = _saturate(srv, sat_sids, a, pool, frame_idx)
    srv.set_inflight(2)
    for sid, _ in sat_sids:
        srv.close_session(sid)
    srv.close()

    # the plain FP32 path, one session at a time, same frames
    plain_s = 0.0
    plain_evals = 0.0
    lat_plain = [0.0]
    plain_by_session = []
    for spec in ([] if a.no_plain else specs):
        f = g.Filter(spec["P"], spec["K"], spec["N"], seed=spec["seed"])
        _setup_session(f, pool, spec, dev)
        torch.cuda.synchronize()
        for i in range(len(spec["arrivals"])):
            fi = frame_idx(spec, i)
            ts = time.perf_counter()
            f.step(pool["scans"][fi][:spec["N"]], pool["odometry"][fi], pool["cov"])
            dt = time.perf_counter() - ts
            plain_s += dt
            lat_plain.append(dt)
            plain_evals += spec["P"] * spec["N"] * 3
            plain_by_session.append((spec, dt))
        f.close()
    served_rate = stats["evals"] / stats["span_s"] if stats["span_s"] > 0 else 0.0
    # latency by session size: frames of the smallest and the largest quarter of the
    # sessions (by particles x points), to show how much a small frame waits for large ones
    works = np.array(sorted({sp["P"] * sp["N"] for sp in specs}))
    q1, q3 = np.percentile(works, 25), np.percentile(works, 75)
    small = np.array([l for wk, l in lat_by_work if wk <= q1]) * 1e3
    large = np.array([l for wk, l in lat_by_work if wk >= q3]) * 1e3
    by_size = {"small_quarter": {"p50": float(np.percentile(small, 50)), "p99": float(np.percentile(small, 99)),
                                 "frames": int(small.size), "max_particles_x_points": float(q1)} if small.size else None,
               "large_quarter": {"p50": float(np.percentile(large, 50)), "p99": float(np.percentile(large, 99)),
                                 "frames": int(large.size), "min_particles_x_points": float(q3)} if large.size else None}
    if small.size and large.size:
        by_size["small_over_large_p50"] = by_size["small_quarter"]["p50"] / by_size["large_quarter"]["p50"]
    sat_ids = {sp["seed"] for _, sp in sat_sids}
    sat_plain = [(spec, t) for spec, t in plain_by_session if spec["seed"] in sat_ids]
    sat_plain_rate = (sum(sp["P"] * sp["N"] * 3 for sp, _ in sat_plain) / sum(t for _, t in sat_plain)
                      if sat_plain else None)
    return {
        "metric": "serving: aggregate particle×point lik+grad evals/s and p50/p99 frame latency",
        "value": served_rate, "unit": "evals/s", "n_gpus": 1, "higher_is_better": True,
        "config": {"workload": f"{len(specs)} sessions, P~U[4096,200000], N~U[1024,8192], K~U[10,300], "
                               f"{a.session_frames} Poisson frames at {a.serve_rate:g} Hz each, {a.budget_gb:.0f} GB budget, "
                               f"{a.serve_dtype.upper()} tables, scenes to {a.serve_range:.0f} m",
                   "sessions": len(specs), "frames": stats["frames"]},
        "latency_ms": {"p50": stats["latency_p50_s"] * 1e3, "p99": stats["latency_p99_s"] * 1e3,
                       "max": stats["latency_max_s"] * 1e3, "mean": stats["latency_mean_s"] * 1e3,
                       "measured": "submission to completion (server clock)"},
        "latency_by_session_size_ms": by_size, "tick_work_cap": a.tick_work,
        "latency_from_arrival_ms": {"p50": float(np.percentile(e2e_lat, 50)) * 1e3,
                                    "p99": float(np.percentile(e2e_lat, 99)) * 1e3,
                                    "measured": "scheduled Poisson arrival to completion"},
        "mean_sessions_per_tick": stats["mean_sessions_per_tick"], "ticks": stats["ticks"],
        "gpu_busy_s": stats["busy_s"], "evals_per_gpu_busy_s": stats["evals"] / stats["busy_s"] if stats["busy_s"] else None,
        "saturated": {"sessions": len(sat_sids),
                      "two_ticks_in_flight_evals_per_s": sat[2]["evals"] / sat[2]["span_s"] if sat[2]["span_s"] else None,
                      "one_tick_in_flight_evals_per_s": sat[1]["evals"] / sat[1]["span_s"] if sat[1]["span_s"] else None,
                      "mean_sessions_per_tick": [sat[2]["mean_sessions_per_tick"], sat[1]["mean_sessions_per_tick"]],
                      "plain_fp32_same_sessions_evals_per_s": sat_plain_rate},

        "wall_s": wall, "session_setup_s": setup_s, "generation_s": t_gen,
        "plain_fp32_one_at_a_time": {"evals_per_s": plain_evals / plain_s if plain_s else None,
                                     "frame_ms_p50": float(np.percentile(lat_plain, 50)) * 1e3,
                                     "frame_ms_p99": float(np.percentile(lat_plain, 99)) * 1e3, "busy_s": plain_s},
        "offered_evals_per_s": float(np.mean([s["P"] * s["N"] * 3 for s in specs]) * a.serve_rate * len(specs)),
        "rate_hz_per_session": a.serve_rate,
    }


# ----------------------------------------------------------------------------- reference arm (the oracle)
def run_reference(a, world, rank):
    """The FP64 oracle as the reference implementation, on the host cores: each
    step is one whole frame on a bounded particle sample of the same session."""
    if rank != 0:
        return None
    import synth
    cores = max(1, min(host_cores(), 64))
    per = max(16, min(64, a.particles // cores))
    frames = a.warmup + a.steps
    w = synth.forest_workload(seed=0, n_particles=per * cores, n_points=a.points, n_keyframes=a.keyframes,
                              n_frames=frames)
    opool = OraclePool(w, per * cores)
    times = np.array([opool.frame(fr)[0] for fr in range(frames)])[a.warmup:]
    opool.close()
    P_s = opool.per_worker * opool.workers
    N = a.points
    value = P_s * N * 3 * len(times) / times.sum()
    desc = (f"FP64 oracle, whole frame per step on {P_s} particles of the session: {opool.workers} forked "
            f"workers (one per host core) with {opool.per_worker} particles each ({N} points, "
            f"{a.keyframes} keyframes, 3 moves)")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": float(times.mean()) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"single session, {a.particles} particles x {N}-point scans x "
                                   f"{a.keyframes} keyframes; each step a {P_s}-particle sample",
                       "particles": a.particles, "points": N, "keyframes": a.keyframes},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": opool.workers, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    world, rank, local = dist_env()
    if a.impl == "reference":
        line = run_reference(a, world, rank)
    elif a.serve:
        line = run_serve(a) if rank == 0 else None
    else:
        line = run_native(a, world, rank, local)
    if rank == 0 and line is not None:
        s = json.dumps(line)
        print(s, flush=True)
        if a.out:
            with open(a.out, "w") as fh:
                fh.write(s + "\n")


if __name__ == "__main__":
    main()

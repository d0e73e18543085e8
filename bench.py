#!/usr/bin/env python3
"""MM-BA throughput benchmark: LM iterations per second on the city-scale scene.

One step is one Levenberg-Marquardt iteration of the MM bundle adjustment on
the whole problem: per-scan damped 6x6 solves and retraction, the trial voxel
pass (posed covariance, 3x3 eigen-solve and cost of every voxel), the device
decision, and on acceptance the scan pass (surrogate gradient and Hessian).
Timed steps run as solves of --iters-per-solve iterations from the perturbed
initial poses (the state is reset between solves, outside the timed region),
so the accepted/rejected mix is that of a real solve.

Workload (default "city"): 10,000 scans, 500,000 planar voxels, 10-50
observations each (~15M point clusters), 32 points per observation, built on
the GPU from raw points.  Under torchrun each rank solves its own independent
scene (weak scaling, no collective on the data path).

--impl reference times the CPU oracle (plain sequential FP64 C) on a bounded
sample of the same workload and scales to the full problem.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MM-BA iter/s & plane-obs/s @10k scans; served jobs/s, p99 vs plain FP64"
HBM_PEAK_FALLBACK = 6800.0
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (non-tensor and tensor alike)
# FP64 voxel pass: floating-point operations per observation in the kernel
# (an FMA counts as 2), with the scatter as its pivoted LDL^T: q = R m + t
# (18), q - a (3), the columns W of R P^T L (18), D-weighted columns and
# N (q - a) (12), accumulation of M (48), sums of N (q - a) and N (4).
VOXEL_PASS_FLOP_PER_OBS = 103
# bytes one voxel-pass launch must move per observation slot: 10 doubles + a
# 4-byte scan index (the pose table and per-voxel outputs are small)
VOXEL_PASS_BYTES_PER_ELEM = 84
# The method's bytes of one mixed voxel pass (the roofline's numerator): per
# observation its cluster, 10 FP32 values, and a 4-byte scan index; per voxel
# its observation count (4 B) and a 32-byte plane record written.
MIXED_ALG_BYTES_PER_OBS = 44
MIXED_ALG_BYTES_PER_VOXEL = 36
# What this layout moves per launch (reported beside it): per observation one
# 48-byte slot (offset and N, scatter eigenvalues and scan index, eigenvector
# quaternion); per voxel its length (4 B), anchor (16 B), frame and centroid
# read and written (2 x 32 B) and the plane written (16 B)
MIXED_VOXEL_BYTES_PER_OBS = 48
MIXED_VOXEL_BYTES_PER_VOXEL = 100


def _args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000, help="timed LM iterations per rank")
    ap.add_argument("--warmup", type=int, default=30, help="untimed warm-up iterations")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["city", "mid", "tiny", "batched", "served", "voxelize", "sweep"],
                    default="city")
    ap.add_argument("--batched-jobs", type=int, default=256, help="jobs of the batched workload")
    ap.add_argument("--fp64-jobs", type=int, default=256, help="batched: of which solved on the plain FP64 path too")
    ap.add_argument("--served-jobs", type=int, default=20000, help="jobs of the served stream")
    ap.add_argument("--served-fp64-jobs", type=int, default=200,
                    help="served: the stream's first arrivals also served by the plain FP64 path")
    ap.add_argument("--burst-jobs", type=int, default=2000, help="served: jobs of the capacity burst")
    ap.add_argument("--agreement-jobs", type=int, default=16, help="batched: jobs of the pose-agreement study")
    ap.add_argument("--cpu-jobs", type=int, default=20, help="batched / served: jobs timed on the CPU oracle")
    ap.add_argument("--gen-priority", type=int, default=-5,
                    help="served: CUDA priority of the job generator's stream (lower is higher; clamped)")
    ap.add_argument("--no-batched", action="store_true", help="default run: skip the batched workload")
    ap.add_argument("--no-served", action="store_true", help="default run: skip the served workload")
    ap.add_argument("--no-voxelize", action="store_true", help="default run: skip the preprocessing workload")
    ap.add_argument("--rate", type=float, default=200.0, help="served: Poisson arrival rate (jobs/s)")
    ap.add_argument("--loaders", type=int, default=3, help="served: the server's loader threads")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="served: device memory budget")
    ap.add_argument("--chunk", type=int, default=0,
                    help="batched / served: LM iterations per round (0: 8 batched, 16 served)")
    ap.add_argument("--iters-per-solve", type=int, default=30)
    ap.add_argument("--e2e-jobs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU budget of the oracle baseline")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--fp64-steps", type=int, default=60,
                    help="iterations of the plain FP64 path timed for comparison (0: skip)")
    ap.add_argument("--shrink", type=float, default=1.0,
                    help="scale scans, voxels and area by this factor at equal density (profiling runs)")
    return ap.parse_args()


WORKLOAD_TEXT = {
    "city": "city: 10,000 scans, 500,000 planar voxels, 10-50 obs/voxel (~15M point clusters), 32 pts/obs, "
            "patch 0.5-4 m log-uniform, 5% strips, 2 cm noise, 0.5 deg / 10 cm perturbation, 2x2 km slab",
    "mid": "mid: 1,000 scans, 50,000 voxels, 8-40 obs/voxel (~1.2M clusters), 100 pts/obs",
    "tiny": "tiny: 20 scans, 200 voxels, 5-20 obs/voxel, 50 pts/obs",
}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.lines = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons, n = [], [], set(), 0
        for ts, line in self.lines:
            if not (t0 - 0.2 <= ts <= t1 + 0.2):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            n += 1
            for name, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


def _gpu_id(torch, dev: int) -> str | None:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def workload_config(args, scene, world):
    """The workload a line is measured on (the same for both arms)."""
    gb = MIXED_ALG_BYTES_PER_OBS * scene.n_obs / 1e9
    l2 = (f"inputs larger than L2 (every pass streams {gb:.2f} GB of clusters)" if gb > 0.129 else
          f"inputs of {gb:.3f} GB fit in L2 (no flush: not a timing-rule workload)")
    return {"workload": WORKLOAD_TEXT[args.workload], "n_scans": scene.n_scans, "n_voxels": scene.n_voxels,
            "n_obs": scene.n_obs, "l2": l2, "parallelism": f"{world} independent job(s), one per GPU"}


def scene_params(scenegen, args, rank):
    p = scenegen.config(args.workload, rep=rank)
    if args.shrink != 1.0:
        f = args.shrink
        side = math.sqrt(f)
        p = scenegen.replace(p, n_scans=max(1, int(p.n_scans * f)), n_voxels=max(1, int(p.n_voxels * f)),
                             box=(p.box[0] * side, p.box[1] * side, p.box[2]))
    return p


def device_clusters(scene, torch, mm, chunk_obs: int = 1 << 20):
    """Raw points generated on the host in chunks, clustered on the GPU."""
    import numpy as np
    dev = torch.device("cuda")
    n_obs, npo = scene.n_obs, scene.params.pts_per_obs
    agg = torch.empty((n_obs, 10), dtype=torch.float64, device=dev)
    host = torch.empty((min(chunk_obs, n_obs) * npo, 3), dtype=torch.float64).pin_memory()
    hnp = host.numpy()
    for o0 in range(0, n_obs, chunk_obs):
        o1 = min(n_obs, o0 + chunk_obs)
        n = o1 - o0
        scene.points(o0, o1, out=hnp[: n * npo])
        pts = host[: n * npo].to(dev, non_blocking=True)
        po = torch.arange(n + 1, dtype=torch.int64, device=dev) * npo
        mm.ba_aggregate_points(po, pts, agg[o0:o1], stream=torch.cuda.current_stream())
        torch.cuda.current_stream().synchronize()
    return agg


def device_clusters_gpu(scene, torch, mm, chunk_obs: int = 1 << 20):
    """Raw points generated on the GPU in chunks, clustered on the GPU."""
    dev = torch.device("cuda")
    n_obs, npo = scene.n_obs, scene.params.pts_per_obs
    agg = torch.empty((n_obs, 10), dtype=torch.float64, device=dev)
    buf = torch.empty((min(chunk_obs, n_obs) * npo, 3), dtype=torch.float64, device=dev)
    for o0 in range(0, n_obs, chunk_obs):
        o1 = min(n_obs, o0 + chunk_obs)
        n = o1 - o0
        pts = buf[: n * npo]
        scene.points_device(o0, o1, pts)
        po = torch.arange(n + 1, dtype=torch.int64, device=dev) * npo
        mm.ba_aggregate_points(po, pts, agg[o0:o1], stream=torch.cuda.current_stream())
    del buf
    return agg


def job_params(scenegen, k, scans_min, scans_max, base_seed):
    """One job of the many-job workloads: scans log-uniform in [min, max],
    voxels = 50 x scans, 5-30 observations per voxel, 32 points each, 2 cm
    noise, 0.5 deg / 10 cm initial perturbation, patches in a 50 m cube."""
    import numpy as np
    rng = np.random.default_rng(base_seed + k)
    n_scans = int(round(math.exp(rng.uniform(math.log(scans_min), math.log(scans_max)))))
    return scenegen.SceneParams(n_scans=n_scans, n_voxels=50 * n_scans, obs_min=5, obs_max=30, pts_per_obs=32,
                                noise_sigma=0.02, rot_sigma_deg=0.5, trans_sigma=0.10, seed=base_seed + k)


def kernel_source_hash(kernel: str = "voxel_pass_f64") -> str:
    h = hashlib.sha256()
    main = "voxelize.cu" if kernel.startswith("l1_") else "iter_mixed.cu" if "mixed" in kernel else "iter_f64.cu"
    for f in (main, "mmba_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2608_14266_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec.get(kernel, {})
        if e.get("source_hash") == kernel_source_hash(kernel) and workload in e.get("bytes_per_launch", {}):
            return e["bytes_per_launch"][workload]
    except (OSError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample(scene, budget_s: float, min_obs: int = 20000):
    """A prefix of the voxels with their clusters (oracle-formed), sized so
    that one oracle LM iteration takes roughly budget_s seconds."""
    import numpy as np

    import oracle
    rate = 3.0e6  # rough oracle speed (cluster-iterations per second), refined below
    target = int(max(min_obs, min(scene.n_obs, rate * budget_s)))
    nv = int(np.searchsorted(scene.voxel_off, target, side="right")) - 1
    nv = max(1, min(scene.n_voxels, nv))
    n_obs = int(scene.voxel_off[nv])
    pts = scene.points(0, n_obs)
    cen = oracle.points_to_centred(np.arange(n_obs + 1, dtype=np.int64) * scene.params.pts_per_obs, pts)
    prob = oracle.ObsProblem(scene.n_scans, scene.voxel_off[: nv + 1], scene.obs_scan[:n_obs], cen)
    return prob, nv


def time_oracle(scene, steps: int, warmup: int, total_budget_s: float, all_cores: bool = False):
    """Times oracle LM iterations on a bounded sample; returns the full-problem
    iterations per second and the description of the sample (and, with
    all_cores, the same sample's iteration on every host core)."""
    import oracle
    per_step = max(0.05, total_budget_s / max(1, steps + warmup))
    prob, nv = oracle_sample(scene, per_step)
    lm = oracle.LM(prob, scene.pose_init)
    for _ in range(warmup):
        lm.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        lm.step()
    dt = (time.perf_counter() - t0) / max(1, steps)
    frac = prob.n_obs / scene.n_obs
    sample = (f"first {nv} of {scene.n_voxels} voxels ({prob.n_obs} of {scene.n_obs} clusters, "
              f"{100 * frac:.2f}%), {steps} oracle LM iterations after {warmup} warm-up, "
              f"time scaled by clusters to the full problem")
    if not all_cores:
        return frac / dt, dt, sample
    dt_par, threads = time_oracle_threads(prob, scene.pose_init, steps, warmup)
    par = {"value": frac / dt_par, "unit": "iter/s", "cores": threads, "kind": "oracle",
           "sample": sample.replace("oracle LM iterations", "oracle iterations (voxel and g, H terms over voxel "
                                    "segments, one thread per core; per-scan solves and retractions)")}
    return frac / dt, dt, sample, par


def time_oracle_threads(prob, poses, steps: int, warmup: int):
    """The oracle's iteration on every host core: the voxels split into
    contiguous segments of equal observation count, one thread per segment
    evaluating the cost terms and the per-scan g, H (the oracle's C calls
    release the interpreter lock), the sums added, then the damped per-scan
    solves and retractions split over the threads.  Returns seconds per
    iteration and the thread count."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    T = max(1, os.cpu_count() or 1)
    vo = prob.voxel_off
    cuts = np.unique(np.searchsorted(vo, np.linspace(0, prob.n_obs, T + 1)[1:-1]))
    edges = [0] + [int(c) for c in cuts if 0 < c < prob.n_voxels] + [prob.n_voxels]
    segs = [oracle.ObsProblem(prob.n_scans, vo[a:b + 1] - vo[a], prob.obs_scan[vo[a]:vo[b]], prob.agg[vo[a]:vo[b]])
            for a, b in zip(edges[:-1], edges[1:]) if b > a]
    scans = np.array_split(np.arange(prob.n_scans), T)
    P = np.ascontiguousarray(poses, dtype=np.float64)

    def terms(seg):
        c, planes = oracle.voxel_pass(seg, P)
        g, H = oracle.grad_hess(seg, P, planes)
        return c, g, H

    def solve(js, g, H, out):
        for j in js:
            A = H[j] + oracle.DEFAULT_MU0 * np.diag(np.diag(H[j]))
            rc, d = oracle.ldlt6(A, -g[j])
            out[j] = oracle.retract(P[j], d if rc == 0 else np.zeros(6))

    with ThreadPoolExecutor(T) as pool:
        def iteration():
            parts = list(pool.map(terms, segs))
            g = sum(p[1] for p in parts)
            H = sum(p[2] for p in parts)
            out = np.empty_like(P)
            list(pool.map(lambda js: solve(js, g, H, out), scans))
            return out
        for _ in range(warmup):
            iteration()
        t0 = time.perf_counter()
        for _ in range(steps):
            iteration()
        return (time.perf_counter() - t0) / max(1, steps), T


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import scenegen
    scene = scenegen.make_scene(scene_params(scenegen, args, 0))
    budget = 150.0
    ips, dt, sample, par = time_oracle(scene, args.steps, args.warmup, budget, all_cores=True)
    line = {
        "impl": "reference", "metric": METRIC, "value": ips, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / ips, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene generator)",
        "config": workload_config(args, scene, 1),
        "run": {"solver": "CPU oracle, FP64", "iters_per_solve": args.iters_per_solve},
        "plane_obs_per_s": ips * scene.n_obs,
        "e2e": {"value": ips, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": ips, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "all_cores": par},
    }
    print(json.dumps(line), flush=True)


def measure(mm, torch, scene, dev_inputs, precision, steps, warmup, S, barrier, local, profile=True):
    """Times `steps` LM iterations (solves of S iterations from the initial
    poses, state reset outside the timed region) with CUDA events on the
    library's stream; returns the timing, the kernel breakdown and clocks.

    The timed pass records no event between the iteration's launches (each
    event record between two kernels adds its own gap, ~4 us per launch);
    with profile=True a second timed pass of the same steps brackets every
    launch with events for the per-kernel times."""
    voxel_off, obs_scan, agg, pose0 = dev_inputs
    stream = torch.cuda.current_stream()
    ba = mm.BundleAdjuster(cuda_stream=stream, precision=precision)
    ba.load_observations(scene.n_scans, voxel_off, obs_scan, agg, pose0)
    cfg = ba.cfg

    def reset():
        ba.set_state(pose0, cfg.mu0, 2.0)

    done = 0
    while done < warmup:
        n = min(S, warmup - done)
        ba.iterate(n, stats=False)
        done += n
        reset()
    torch.cuda.synchronize()
    reps = []
    left = steps
    while left > 0:
        reps.append(min(S, left))
        left -= reps[-1]

    def timed_pass(kernel_events):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in reps]
        accepted = launches = 0
        acc0 = ba.stats()["accepted"]
        ba.profile(kernel_events)
        for (e0, e1), n in zip(ev, reps):
            barrier()
            torch.cuda.synchronize()
            l0 = ba.kernel_launches()
            e0.record(stream)
            ba.iterate(n, stats=False)
            e1.record(stream)
            launches += ba.kernel_launches() - l0
            torch.cuda.synchronize()
            acc1 = ba.stats()["accepted"]
            accepted += acc1 - acc0
            reset()
            acc0 = ba.stats()["accepted"]
        torch.cuda.synchronize()
        prof = ba.profile_read() if kernel_events else None
        ba.profile(False)
        return sum(e0.elapsed_time(e1) for e0, e1 in ev), accepted, launches, prof

    clocks = ClockSampler(_gpu_id(torch, local)) if profile else None
    if profile:
        time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed")
    t_wall0 = time.time()
    ms, accepted, launches, _ = timed_pass(False)
    t_wall1 = time.time()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop(t_wall0, t_wall1) if clocks else None
    prof, ms_events = None, None
    if profile:
        ms_events, _, _, prof = timed_pass(True)
    ba.close()
    return {"ms": ms, "accepted": accepted, "launches": launches, "prof": prof, "clocks": clk,
            "ms_with_kernel_events": ms_events}


def roofline_for(precision, scene, prof, workload):
    vp_ms, vp_n = prof["voxel_pass"]
    vp_avg_s = vp_ms / max(1, vp_n) / 1000.0
    if precision == "fp64":
        flops = VOXEL_PASS_FLOP_PER_OBS * scene.n_obs
        achieved = flops / vp_avg_s / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": recorded_traffic(workload, "voxel_pass_f64"),
                "kernel": "voxel_pass_f64", "avg_launch_ms": vp_avg_s * 1000.0,
                "peak_source": "nominal GB300 FP64 rate (the measured peaks have no FP64 entry)",
                "flop_per_launch": flops,
                "hbm_view_gbs": VOXEL_PASS_BYTES_PER_ELEM * scene.n_obs / vp_avg_s / 1e9}
    peak, src = hbm_peak()
    nbytes = MIXED_ALG_BYTES_PER_OBS * scene.n_obs + MIXED_ALG_BYTES_PER_VOXEL * scene.n_voxels
    layout = MIXED_VOXEL_BYTES_PER_OBS * scene.n_obs + MIXED_VOXEL_BYTES_PER_VOXEL * scene.n_voxels
    achieved = nbytes / vp_avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(workload, "voxel_pass_mixed"), "kernel": "voxel_pass_mixed",
            "avg_launch_ms": vp_avg_s * 1000.0, "peak_source": src, "bytes_per_launch": nbytes,
            "basis": "the method's bytes: 44 B per observation (10 FP32 cluster values + scan index) + "
                     "36 B per voxel (count + 32-byte plane record)",
            "layout_bytes_per_launch": layout, "layout_gbs": layout / vp_avg_s / 1e9}


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return HBM_PEAK_FALLBACK, "fallback 6.8 TB/s"


def run_ours(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    import scenegen

    from paper_2608_14266_gb300 import replicas
    rank, world, local = replicas.rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    group = replicas.Group(dist, torch.device("cuda", local))
    barrier, max_over_ranks = group.barrier, group.max

    scene = scenegen.make_scene(scene_params(scenegen, args, replicas.scene_rep(rank)))
    dev = torch.device("cuda", local)
    agg = device_clusters(scene, torch, mm)
    inputs = (torch.from_numpy(scene.voxel_off).to(dev), torch.from_numpy(scene.obs_scan).to(dev), agg,
              torch.from_numpy(scene.pose_init).to(dev))
    S = args.iters_per_solve
    prec = mm.BA_MIXED if args.precision == "mixed" else mm.BA_FP64
    res = measure(mm, torch, scene, inputs, prec, args.steps, args.warmup, S, barrier, local)
    ms = max_over_ranks(res["ms"])
    value = args.steps * world / (ms / 1000.0)
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        r64 = measure(mm, torch, scene, inputs, mm.BA_FP64, args.fp64_steps, min(args.warmup, S), S, barrier,
                      local, profile=False)
        ms64 = max_over_ranks(r64["ms"])
        fp64 = {"value": args.fp64_steps * world / (ms64 / 1000.0), "unit": "iter/s", "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps, "accepted_iters": r64["accepted"]}

    # end to end through the public API with pinned host buffers
    agg_h = torch.empty(agg.shape, dtype=torch.float64).pin_memory()
    agg_h.copy_(agg)
    vo_h = torch.from_numpy(scene.voxel_off).pin_memory()
    os_h = torch.from_numpy(scene.obs_scan).pin_memory()
    p0_h = torch.from_numpy(scene.pose_init).pin_memory()
    out_h = torch.empty((scene.n_scans, 12), dtype=torch.float64).pin_memory()
    del agg, inputs
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    e2e_times, e2e_phase = [], {"load_ms": 0.0, "iterate_and_read_ms": 0.0}
    for k in range(args.e2e_jobs + (1 if args.e2e_jobs else 0)):  # the first job is an untimed warm-up
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mm.BundleAdjuster(cuda_stream=stream, precision=prec) as job:
            job.load_observations(scene.n_scans, vo_h.numpy(), os_h.numpy(), agg_h.numpy(), p0_h.numpy())
            stream.synchronize()
            t1 = time.perf_counter()
            job.iterate(S, stats=False)
            job.poses(out=out_h.numpy())
            t2 = time.perf_counter()
        if k == 0:
            continue
        e2e_times.append(time.perf_counter() - t0)
        e2e_phase["load_ms"] += (t1 - t0) * 1e3 / args.e2e_jobs
        e2e_phase["iterate_and_read_ms"] += (t2 - t1) * 1e3 / args.e2e_jobs
    e2e_phase["job_ms"] = [round(t * 1e3, 3) for t in e2e_times]
    e2e_value = None
    if e2e_times:
        e2e_value = world * S * args.e2e_jobs / max_over_ranks(sum(e2e_times))
        # where the load time goes: the same load from device-resident inputs,
        # and a plain pinned host-to-device copy of the clusters
        vo_d, os_d, agg_d, p0_d = (vo_h.to(dev), os_h.to(dev), agg_h.to(dev), p0_h.to(dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mm.BundleAdjuster(cuda_stream=stream, precision=prec) as job:
            job.load_observations(scene.n_scans, vo_d, os_d, agg_d, p0_d)
            stream.synchronize()
            e2e_phase["load_from_device_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        agg_d.copy_(agg_h, non_blocking=True)
        torch.cuda.synchronize()
        e2e_phase["h2d_copy_gbs"] = agg_h.numel() * 8 / (time.perf_counter() - t0) / 1e9
        del vo_d, os_d, agg_d, p0_d
    h2d = agg_h.numel() * 8 + vo_h.numel() * 8 + os_h.numel() * 4 + p0_h.numel() * 8
    d2h = out_h.numel() * 8

    prof = res["prof"]
    roofline = roofline_for(args.precision, scene, prof, args.workload)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        ips, dt, sample, par = time_oracle(scene, 2, 1, args.cpu_seconds, all_cores=True)
        cpu = {"value": ips, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": sample, "all_cores": par}
    per_obs = MIXED_VOXEL_BYTES_PER_OBS if args.precision == "mixed" else VOXEL_PASS_BYTES_PER_ELEM
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded scene generator; points clustered on GPU)",
        "config": workload_config(args, scene, world),
        "run": {"precision": args.precision, "iters_per_solve": S, "accepted_iters": res["accepted"],
                "per_pass_cluster_gb": round(scene.n_obs * per_obs / 1e9, 3)},
        "plane_obs_per_s": value * scene.n_obs,
        "fp64_path": fp64,
        "clocks": res["clocks"],
        "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": h2d / S, "d2h_bytes_per_step": d2h / S,
                "jobs": args.e2e_jobs, "per_job": e2e_phase,
                "scope": "ba_load_observations (pinned host clusters) + "
                                                f"{S} iterations + ba_poses to host, per job, after one untimed "
                                                "warm-up job"},
        "gpu_launches": int(res["launches"]),
        "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items()},
        "kernel_events": {"pass": "a second timed pass of the same steps with events around every launch "
                                  "(the kernel_ms and the roofline's launch times)",
                          "ms_per_step": res["ms_with_kernel_events"] / args.steps},
        "roofline": roofline,
        "cpu_baseline": cpu,
    }
    # configs 4 and 5 and the preprocessing (one GPU): nested in the same line
    if world == 1:
        import oracle
        ora = None if args.no_cpu_baseline else oracle
        if not args.no_batched:
            line["batched"] = batched_result(args, mm, torch, scenegen, ora)
        if not args.no_served:
            line["served"] = served_result(args, mm, torch, scenegen, ora)
        if not args.no_voxelize:
            line["voxelize"] = voxelize_result(args, mm, torch, scenegen)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _gt_rms(P, gt):
    """RMS rotation (rad) and translation (m) error of solved poses against
    the generator's ground truth gt (scan 0, the gauge, is exact on both)."""
    import numpy as np
    R1 = P[:, :9].reshape(-1, 3, 3)
    R2 = gt[:, :9].reshape(-1, 3, 3)
    D = np.einsum("nij,nkj->nik", R1, R2)
    ang = np.arccos(np.clip(0.5 * (np.trace(D, axis1=1, axis2=2) - 1.0), -1.0, 1.0))
    return float(np.sqrt(np.mean(ang ** 2))), float(np.sqrt(np.mean(np.sum((P[:, 9:] - gt[:, 9:]) ** 2, 1))))


class _Accuracy:
    """Per-path mean over jobs of the RMS error against ground truth."""

    def __init__(self):
        self.sums = {}

    def add(self, path, P, gt):
        r, t = _gt_rms(P, gt)
        a = self.sums.setdefault(path, [0.0, 0.0, 0])
        a[0] += r
        a[1] += t
        a[2] += 1

    def report(self):
        return {k: {"rms_rot_rad": v[0] / v[2], "rms_trans_m": v[1] / v[2], "jobs": v[2]} for k, v in self.sums.items()}


def _pose_diff(P, Q):
    import numpy as np
    R1 = P[:, :9].reshape(-1, 3, 3)
    R2 = Q[:, :9].reshape(-1, 3, 3)
    D = np.einsum("nij,nkj->nik", R1, R2)
    ang = np.arctan2(0.5 * np.linalg.norm(np.stack([D[:, 2, 1] - D[:, 1, 2], D[:, 0, 2] - D[:, 2, 0],
                                                    D[:, 1, 0] - D[:, 0, 1]], 1), axis=1),
                     0.5 * (np.trace(D, axis1=1, axis2=2) - 1.0))
    return float(ang.max()), float(np.abs(P[:, 9:] - Q[:, 9:]).max())


SOLVE_CFG = dict(rel_tol=1e-8, max_iters=200, max_consec_reject=10)


class JobFactory:
    """Jobs of the many-job workloads generated on the GPU, all queued on one
    stream: structure, poses and patches by the scene generator's device
    kernels (the host generator's streams), points drawn in FP32 from the same
    per-observation counters (scenegen_gpu.cu), clusters formed by the
    library (ba_aggregate_points)."""

    def __init__(self, mm, torch, stream, chunk_obs: int = 1 << 20, pts_per_obs: int = 32):
        self.mm, self.torch, self.stream = mm, torch, stream
        self.chunk, self.npo = chunk_obs, pts_per_obs
        with torch.cuda.stream(stream):
            self.buf = torch.empty((chunk_obs * pts_per_obs, 3), dtype=torch.float64, device="cuda")
            self.po = torch.arange(chunk_obs + 1, dtype=torch.int64, device="cuda") * pts_per_obs

    host_s = {"structure": 0.0, "clusters": 0.0}  # host time spent queueing the work

    def make(self, params, offsets=None):
        import scenegen
        assert params.pts_per_obs == self.npo
        torch = self.torch
        t0 = time.perf_counter()
        sc = scenegen.make_scene_device(params, stream=self.stream, offsets=offsets)
        t1 = time.perf_counter()
        with torch.cuda.stream(self.stream):
            agg = torch.empty((max(sc.n_obs, 1), 10), dtype=torch.float64, device="cuda")[: sc.n_obs]
        for o0 in range(0, sc.n_obs, self.chunk):
            o1 = min(sc.n_obs, o0 + self.chunk)
            pts = self.buf[: (o1 - o0) * self.npo]
            sc.points_fast(o0, o1, pts, stream=self.stream)
            self.mm.ba_aggregate_points(self.po[: o1 - o0 + 1], pts, agg[o0:o1], stream=self.stream)
        self.host_s = {"structure": self.host_s["structure"] + (t1 - t0),
                       "clusters": self.host_s["clusters"] + (time.perf_counter() - t1)}
        return sc, agg


def _dev_inputs(sc, agg):
    return sc.voxel_off, sc.obs_scan, agg, sc.pose_init


def _oracle_seconds_per_job(oracle_mod, samples):
    """Oracle seconds per job on a sample: one timed oracle LM iteration per
    job (after its set-up), times the iterations the plain FP64 GPU path
    needed for that job.  samples: (n_scans, voxel_off, obs_scan, agg, poses,
    iterations) on the host."""
    per_job = []
    for n_scans, vo, os_, ag, po, iters in samples:
        lm = oracle_mod.LM(oracle_mod.ObsProblem(n_scans, vo, os_, ag), po)
        t0 = time.perf_counter()
        lm.step()
        per_job.append((time.perf_counter() - t0) * max(1, iters))
    return float(sum(per_job) / len(per_job))


def _host_sample(sc, agg, iters):
    return (sc.n_scans, sc.voxel_off.cpu().numpy(), sc.obs_scan.cpu().numpy(), agg.cpu().numpy(),
            sc.pose_init.cpu().numpy(), iters)


def _pose_agreement(mm, torch, items, stream):
    """Mixed against plain FP64 poses three ways, on jobs given as (scene,
    clusters) on the device: (a) both paths at the FP64 solve's iteration
    count; (b) both solved to a common tight stop (rel_tol 0: 10 rejected
    steps in a row or 200 iterations); (c) the mixed path stopped by the
    FP64 cost of its own poses (the allocation-free FP64 cost evaluation,
    relative change below 1e-8 on an accepted step), against the FP64 path's
    ordinary stop."""
    worst = {"equal_iterations": [0.0, 0.0], "tight_stop": [0.0, 0.0], "fp64_decided_stop": [0.0, 0.0],
             "default_stop": [0.0, 0.0]}
    iters = {"fp64_default": 0, "mixed_default": 0, "mixed_fp64_decided": 0, "fp64_tight": 0, "mixed_tight": 0}

    def upd(key, P, Q):
        r, t = _pose_diff(P, Q)
        worst[key][0] = max(worst[key][0], r)
        worst[key][1] = max(worst[key][1], t)

    def load(prec, sc, agg, **cfg):
        ba = mm.BundleAdjuster(precision=prec, cuda_stream=stream, **cfg)
        ba.load_observations(sc.n_scans, *_dev_inputs(sc, agg))
        return ba

    for sc, agg in items:
        with load(mm.BA_FP64, sc, agg, **SOLVE_CFG) as b64:
            n64 = b64.solve()["iters"]
            P64 = b64.poses()
        with load(mm.BA_MIXED, sc, agg, **SOLVE_CFG) as bm:
            st = bm.solve()
            upd("default_stop", bm.poses(), P64)
            iters["mixed_default"] += st["iters"]
        iters["fp64_default"] += n64
        with load(mm.BA_MIXED, sc, agg, **SOLVE_CFG) as bm:
            bm.iterate(n64, stats=False)
            upd("equal_iterations", bm.poses(), P64)
        tight = dict(SOLVE_CFG, rel_tol=0.0)
        with load(mm.BA_FP64, sc, agg, **tight) as b64, load(mm.BA_MIXED, sc, agg, **tight) as bm:
            iters["fp64_tight"] += b64.solve()["iters"]
            iters["mixed_tight"] += bm.solve()["iters"]
            upd("tight_stop", bm.poses(), b64.poses())
        # (c): FP64 cost of the mixed iterate after every accepted step
        cost = torch.empty(1, dtype=torch.float64, device="cuda")
        pd = torch.empty((sc.n_scans, 12), dtype=torch.float64, device="cuda")
        with load(mm.BA_MIXED, sc, agg, **tight) as bm:
            prev = None
            n = 0
            while n < SOLVE_CFG["max_iters"]:
                st = bm.iterate(1)
                n += 1
                if not st["last_accepted"]:
                    if st["consec_reject"] >= SOLVE_CFG["max_consec_reject"]:
                        break
                    continue
                bm.poses(out=pd)
                with torch.cuda.stream(stream):
                    mm.ba_eval_cost_noalloc(sc.n_scans, sc.voxel_off, sc.obs_scan, agg, pd, cost, stream=stream)
                c = float(cost.item())
                if prev is None:
                    with torch.cuda.stream(stream):
                        mm.ba_eval_cost_noalloc(sc.n_scans, sc.voxel_off, sc.obs_scan, agg, sc.pose_init, cost,
                                                stream=stream)
                    prev = float(cost.item())
                if prev - c <= SOLVE_CFG["rel_tol"] * prev:
                    break
                prev = c
            iters["mixed_fp64_decided"] += n
            upd("fp64_decided_stop", bm.poses(), P64)
    out = {k: {"max_rot_rad": v[0], "max_trans_m": v[1]} for k, v in worst.items()}
    out["iterations_total"] = iters
    out["jobs"] = len(items)
    return out


def batched_result(args, mm, torch, scenegen, oracle_mod=None):
    """Config 4: many independent jobs solved together in one batch (mixed
    precision, autotuned launch settings, CUDA-graph iterations) against the
    same jobs solved one after another on the plain FP64 path."""
    import numpy as np
    chunk = args.chunk or 8
    n_jobs = args.batched_jobs
    stream = torch.cuda.current_stream()
    params = [job_params(scenegen, k, 20, 2000, 4000) for k in range(n_jobs)]
    fac = JobFactory(mm, torch, stream)
    made = [fac.make(p) for p in params]
    gts = [sc.pose_gt.cpu().numpy() for sc, _ in made]
    torch.cuda.synchronize()
    n_obs = sum(sc.n_obs for sc, _ in made)
    n_vox = sum(sc.n_voxels for sc, _ in made)
    jobs = []
    for sc, agg in made:
        ba = mm.BundleAdjuster(precision=mm.BA_MIXED, cuda_stream=stream, **SOLVE_CFG)
        ba.load_observations(sc.n_scans, *_dev_inputs(sc, agg))
        jobs.append(ba)
    torch.cuda.synchronize()
    with mm.Batch(stream) as b:
        for j in jobs:
            b.add(j)
        t0 = time.perf_counter()
        # the tuner's trials are the solve's first iterations (results do not depend on its choice)
        tune = b.autotune(iters_per_trial=1, passes=1)
        active = b.solve(chunk=chunk)
        torch.cuda.synchronize()
        t_mixed = time.perf_counter() - t0
        launches = b.kernel_launches()
        iters_mixed = sum(j.stats()["iters"] for j in jobs)
        mixed_poses = [j.poses() for j in jobs]
        # roofline of the batch kernels: every job back at its initial poses,
        # four iterations with per-kernel events (every launch covers every job)
        for j, (sc, _) in zip(jobs, made):
            j.set_state(sc.pose_init, 1e-4, 2.0)
        torch.cuda.synchronize()
        b.profile(True)
        b.iterate(4)
        prof = b.profile_read()
        b.profile(False)
    for j in jobs:
        j.close()
    peak, src = hbm_peak()
    vp_ms, vp_n = prof["voxel_pass"]
    vbytes = 4 * (MIXED_ALG_BYTES_PER_OBS * n_obs + MIXED_ALG_BYTES_PER_VOXEL * n_vox)
    achieved = vbytes / (vp_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "voxel_pass_mixed_batch", "avg_launch_ms": vp_ms / max(1, vp_n),
                "launches": vp_n, "peak_source": src,
                "bytes_per_launch": vbytes / max(1, vp_n),
                "basis": "44 B per observation + 36 B per voxel (the method's bytes), all jobs of a group per launch",
                "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items()}}
    # plain FP64, one job after another (loads outside the timed region)
    t_fp64, iters_fp64, worst = 0.0, 0, (0.0, 0.0)
    acc = _Accuracy()
    fp64_iters = []
    n64 = min(n_jobs, args.fp64_jobs)
    for k in range(n64):
        sc, agg = made[k]
        ba = mm.BundleAdjuster(precision=mm.BA_FP64, cuda_stream=stream, **SOLVE_CFG)
        ba.load_observations(sc.n_scans, *_dev_inputs(sc, agg))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ba.solve()
        t_fp64 += time.perf_counter() - t0
        iters_fp64 += st["iters"]
        fp64_iters.append(st["iters"])
        P64 = ba.poses()
        r, t = _pose_diff(mixed_poses[k], P64)
        worst = (max(worst[0], r), max(worst[1], t))
        acc.add("mixed", mixed_poses[k], gts[k])
        acc.add("fp64", P64, gts[k])
        ba.close()
    agreement = _pose_agreement(mm, torch, made[: args.agreement_jobs], stream)
    cpu = None
    if oracle_mod is not None:
        k_s = min(args.cpu_jobs, n64)
        samples = [_host_sample(made[k][0], made[k][1], fp64_iters[k]) for k in range(k_s)]
        s_per_job = _oracle_seconds_per_job(oracle_mod, samples)
        cpu = {"value": 1.0 / s_per_job, "unit": "jobs/s", "cores": 1, "kind": "oracle",
               "sample": f"jobs 0-{k_s - 1} of the batch: one oracle LM iteration each, timed, times the "
                         "iterations the plain FP64 GPU path needed for that job"}
    del made
    torch.cuda.empty_cache()
    return {
        "metric": "batched jobs/s (mixed, one batch) vs sequential plain FP64", "workload": "batched",
        "value": n_jobs / t_mixed, "unit": "jobs/s", "jobs": n_jobs, "clusters": n_obs, "voxels": n_vox,
        "seconds": t_mixed, "iterations": iters_mixed, "unfinished": active, "gpu_launches": launches,
        "fp64_sequential": {"value": n64 / t_fp64 if t_fp64 else None, "unit": "jobs/s", "jobs": n64,
                            "seconds": t_fp64, "iterations": iters_fp64},
        "speedup_vs_fp64": (n_jobs / t_mixed) / (n64 / t_fp64) if t_fp64 else None,
        "pose_agreement_mixed_vs_fp64": {"max_rot_rad": worst[0], "max_trans_m": worst[1], "jobs": n64,
                                         "stop": "each path's own stop rule (rel_tol 1e-8)"},
        "pose_agreement_study": agreement,
        "accuracy_vs_ground_truth": acc.report(),
        "roofline": roofline, "cpu_baseline": cpu,
        "config": {"workload": "256 jobs: scans log-uniform 20-2000, voxels = 50 x scans, 5-30 obs/voxel, "
                               "32 pts/obs, 2 cm noise, 0.5 deg / 10 cm perturbation",
                   "inputs": "each job generated on the GPU (structure, poses, points drawn in FP32, clusters by "
                             "ba_aggregate_points) before the timed region",
                   "stop": SOLVE_CFG, "chunk": chunk,
                   "autotune": {"passes": tune["passes"], "iterations": tune["iterations"],
                                "chosen": tune["candidates"][tune["chosen"]] if tune["chosen"] >= 0 else None,
                                "ms_per_iter": {f"mb{c['min_blocks']}_pf{c['prefetch']}": round(c["ms_per_iter"], 4)
                                                for c in tune["candidates"]}}},
    }


def served_result(args, mm, torch, scenegen, oracle_mod=None):
    """Config 5: an open-loop Poisson stream of BA jobs served by continuous
    batching (mixed precision), each job generated on the GPU from its seed
    when it is admitted, on a side stream, and loaded by the library's loader
    thread while the resident jobs step; against the same stream served one
    job at a time on the plain FP64 path (a stated sample of it)."""
    import collections
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    from paper_2608_14266_gb300.server import Job, Server, latency_summary
    chunk = args.chunk or 16
    n_jobs = args.served_jobs
    rng = np.random.default_rng(77)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=n_jobs))
    params = [job_params(scenegen, k, 50, 5000, 9000) for k in range(n_jobs)]
    main = torch.cuda.current_stream()
    # jobs are generated at the highest priority, so the generator's blocks
    # (partly FP64-bound) share the SMs with the memory-bound iterations
    side = torch.cuda.Stream(priority=args.gen_priority)
    fac = JobFactory(mm, torch, side)
    n_sample = min(n_jobs, args.served_fp64_jobs)
    pool = ThreadPoolExecutor(max(2, min(8, (os.cpu_count() or 2) // 2)))

    def serve(order_arrivals, budget, sample_gt):
        """Serves jobs 0..len(order_arrivals)-1 arriving at the given times."""
        m = len(order_arrivals)
        ahead = collections.deque()
        nxt = 0  # next job whose offsets are requested
        gt_host = {}
        clock0 = time.perf_counter()
        clk = lambda: time.perf_counter() - clock0
        srv = Server(budget, chunk=chunk, clock=clk, precision=mm.BA_MIXED, cuda_stream=main,
                     async_admission=True, input_stream=side, loaders=args.loaders, **SOLVE_CFG)

        def inputs(k, off):
            sc, agg = fac.make(params[k], offsets=off)
            if sample_gt and k < n_sample:
                h = torch.empty((sc.n_scans, 12), dtype=torch.float64).pin_memory()
                with torch.cuda.stream(side):
                    h.copy_(sc.pose_gt, non_blocking=True)
                gt_host[k] = h
            return _dev_inputs(sc, agg)

        k = 0
        prof = {"steps": 0, "step_s": 0.0, "admit_s": 0.0, "resident_sum": 0, "loading_sum": 0}
        srv_admit = srv._admit

        def timed_admit():
            t0 = time.perf_counter()
            n = srv_admit()
            prof["admit_s"] += time.perf_counter() - t0
            return n
        srv._admit = timed_admit
        while k < m or not srv.idle:
            while nxt < m and nxt < k + 64:  # the offsets (count stream, host) of the next arrivals
                ahead.append(pool.submit(scenegen.pinned_voxel_offsets, params[nxt]))
                nxt += 1
            now = clk()
            while k < m and order_arrivals[k] <= now:
                if not ahead:  # a burst ran past the look-ahead
                    ahead.append(pool.submit(scenegen.pinned_voxel_offsets, params[nxt]))
                    nxt += 1
                off = ahead.popleft().result()
                p = params[k]
                srv.submit(Job(job_id=k, n_scans=p.n_scans, n_voxels=p.n_voxels, n_obs=int(off[-1]),
                               arrival=float(order_arrivals[k]), inputs=lambda k=k, off=off: inputs(k, off)))
                k += 1
            if srv.idle:
                time.sleep(max(0.0, min(order_arrivals[k] - now, 0.01)) if k < m else 0.0)
                continue
            t0 = time.perf_counter()
            srv.step()
            prof["step_s"] += time.perf_counter() - t0
            prof["steps"] += 1
            prof["resident_sum"] += len(srv.resident)
            prof["loading_sum"] += len(srv.loading)
        t_end = clk()
        n_st = max(1, prof["steps"])
        host = {"steps": prof["steps"], "step_s": prof["step_s"], "admission_s": prof["admit_s"],
                "generation_queue_s": dict(fac.host_s),
                "mean_resident": prof["resident_sum"] / n_st, "mean_loading": prof["loading_sum"] / n_st}
        fac.host_s = {"structure": 0.0, "clusters": 0.0}
        out = (srv.finished, srv.failed, t_end, srv.kernel_launches(), host)
        srv.close()
        torch.cuda.synchronize()
        return out + (gt_host,)

    budget = args.budget_gb * (1 << 30)
    jobs_m, failed_m, t_m, launches_m, host_m, gt_host = serve(arrivals, budget, True)
    # capacity: a burst of the first jobs all arriving at once
    n_burst = min(n_jobs, args.burst_jobs)
    jobs_b, failed_b, t_b, _, host_b, _ = serve(np.zeros(n_burst), budget, False)
    pool.shutdown()
    torch.cuda.empty_cache()
    # plain FP64, one job at a time, on the first n_sample arrivals of the same stream
    clock0 = time.perf_counter()
    lat64, worst, acc, fp64_iters, samples = [], (0.0, 0.0), _Accuracy(), [], []
    poses_m = {j.job_id: j.poses for j in jobs_m}
    for k in range(n_sample):
        now = time.perf_counter() - clock0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        sc, agg = fac.make(params[k])
        side.synchronize()
        ba = mm.BundleAdjuster(precision=mm.BA_FP64, cuda_stream=main, **SOLVE_CFG)
        ba.load_observations(sc.n_scans, *_dev_inputs(sc, agg))
        st = ba.solve()
        P = ba.poses()
        lat64.append(time.perf_counter() - clock0 - arrivals[k])
        fp64_iters.append(st["iters"])
        gt = gt_host[k].numpy()
        if k in poses_m:
            r, t = _pose_diff(poses_m[k], P)
            worst = (max(worst[0], r), max(worst[1], t))
            acc.add("mixed", poses_m[k], gt)
        acc.add("fp64", P, gt)
        if oracle_mod is not None and len(samples) < args.cpu_jobs:
            samples.append(_host_sample(sc, agg, st["iters"]))
        ba.close()
        del sc, agg
    t64 = time.perf_counter() - clock0
    lat64 = np.array(lat64)
    cpu = None
    if samples:
        s_per_job = _oracle_seconds_per_job(oracle_mod, samples)
        cpu = {"value": 1.0 / s_per_job, "unit": "jobs/s", "cores": 1, "kind": "oracle",
               "sample": f"the stream's first {len(samples)} jobs: one oracle LM iteration each, timed, times "
                         "the iterations the plain FP64 GPU path needed for that job"}
    lat = latency_summary(jobs_m)
    adm = np.array([j.admitted - j.arrival for j in jobs_m if j.admitted is not None])
    iters = np.array([j.stats["iters"] for j in jobs_m])
    value = len(jobs_m) / t_m
    fp64_value = n_sample / t64 if n_sample else None
    return {
        "metric": "served jobs/s and p50/p99 latency (continuous batching, mixed) vs plain FP64 per-job path",
        "workload": "served", "value": value, "unit": "jobs/s", "jobs": n_jobs, "finished": len(jobs_m),
        "failed": len(failed_m), "arrival_rate_per_s": args.rate, "seconds": t_m, "latency": lat,
        "admission_wait_s": {"p50": float(np.percentile(adm, 50)), "p99": float(np.percentile(adm, 99))}
        if adm.size else None,
        "iterations_per_job": {"mean": float(iters.mean()), "max": int(iters.max())} if iters.size else None,
        "capacity_burst": {"value": len(jobs_b) / t_b, "unit": "jobs/s", "jobs": n_burst, "seconds": t_b,
                           "failed": len(failed_b), "latency": latency_summary(jobs_b), "host": host_b},
        "host": host_m,
        "gpu_launches": launches_m,
        "fp64_per_job": None if n_sample == 0 else {
            "value": fp64_value, "unit": "jobs/s", "jobs": n_sample, "seconds": t64,
            "latency": {"p50_s": float(np.percentile(lat64, 50)), "p99_s": float(np.percentile(lat64, 99)),
                        "mean_s": float(lat64.mean()), "max_s": float(lat64.max())},
            "sample": f"the stream's first {n_sample} arrivals, at their arrival times, one job at a time"},
        "speedup_vs_fp64_capacity": (len(jobs_b) / t_b) / fp64_value if fp64_value else None,
        "pose_agreement_mixed_vs_fp64": {"max_rot_rad": worst[0], "max_trans_m": worst[1], "jobs": n_sample,
                                         "stop": "each path's own stop rule (rel_tol 1e-8)"},
        "accuracy_vs_ground_truth": acc.report(),
        "cpu_baseline": cpu,
        "config": {"workload": f"{n_jobs} jobs, Poisson arrivals at {args.rate:g}/s: scans log-uniform 50-5000, "
                               "voxels = 50 x scans, 5-30 obs/voxel, 32 pts/obs, 2 cm noise, 0.5 deg / 10 cm",
                   "budget_gb": args.budget_gb, "chunk": chunk, "stop": SOLVE_CFG,
                   "inputs": "each job generated on the GPU from its seed at admission, on a side stream "
                             "(structure, poses and patches from the generator's streams, points drawn in FP32, "
                             "clusters by ba_aggregate_points); its load and set-up run on the library's loader "
                             "thread and stream while the resident jobs step; the per-job observation counts "
                             "(host count stream, ~1 ms) are drawn by a host thread pool ahead of arrival"},
    }


def _standalone(fn, args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2608_14266_gb300 as mm
    import scenegen
    torch.cuda.set_device(0)
    res = fn(args, mm, torch, scenegen, None if args.no_cpu_baseline else oracle)
    res.setdefault("n_gpus", 1)
    print(json.dumps(res), flush=True)


# preprocessing: FP64 peak from the unit counts (152 SMs x 2 FP64 FMA lanes
# per clock x 2 flops x 2.07 GHz max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# algorithmic work per point of the dominant stages: world point and index
# (9 FMA + 3 adds = 21 flops); the clusters' shifted sums (3 subtractions,
# 3 additions, 6 FMA = 18 flops); the level-1 sort of packed 32-bit keys
# (repack: read 8 B, write 4 B; per 8-bit pass: histogram reads the 4-byte
# key, scatter reads and writes key and value, 4 + 16 B)
VOX_KEYS_FLOPS_PER_POINT = 21
VOX_CLUSTER_FLOPS_PER_POINT = 18
VOX_SORT_BYTES_PER_POINT = lambda passes: 12 + 20 * passes


def run_voxelize(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    import scenegen
    torch.cuda.set_device(0)
    print(json.dumps(voxelize_result(args, mm, torch, scenegen)), flush=True)


def voxelize_result(args, mm, torch, scenegen):
    """Raw scans -> voxels on the device (ba_voxelize: L1 voxelisation, bottom-
    up levels, selection) for the 1,000-scan workload's ~120M points."""
    import numpy as np
    s = scenegen.make_scene(scenegen.config("mid"))
    n_obs, npo = s.n_obs, s.params.pts_per_obs
    P = torch.empty((n_obs * npo, 3), dtype=torch.float64, device="cuda")
    s.points_device(0, n_obs, P)
    order = torch.from_numpy(np.argsort(s.obs_scan, kind="stable")).cuda()
    P = P.view(n_obs, npo, 3)[order].reshape(-1, 3).contiguous()
    counts = np.bincount(s.obs_scan, minlength=s.n_scans) * npo
    spo_h = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n_scans = max(1, int(round(s.n_scans * args.shrink)))  # a prefix of the scans (profiling captures)
    spo_h = spo_h[: n_scans + 1]
    n_pts = int(spo_h[-1])
    P = P[:n_pts].contiguous()
    spo, poses = torch.from_numpy(spo_h).cuda(), torch.from_numpy(s.pose_init[:n_scans]).cuda()
    cfg = dict(voxel_size=0.5, levels=3, tau=0.1, min_obs=2)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        mm.voxelize(spo, P, poses, stream=stream, out="device", **cfg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 10))
    clocks = ClockSampler(_gpu_id(torch, 0))
    time.sleep(0.3)
    stage_ms = {}
    launches = 0
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        v = mm.voxelize(spo, P, poses, stream=stream, out="device", profile=True, **cfg)
        launches += v["launches"]
        for k, x in v["stage_ms"].items():
            stage_ms[k] = stage_ms.get(k, 0.0) + x / steps
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    clk = clocks.stop(t_wall0, t_wall1)
    ms = e0.elapsed_time(e1) / steps
    # end to end: host inputs (pinned) through the same call, results read back to host
    spo_p, P_p, T_p = spo.cpu().pin_memory(), P.cpu().pin_memory(), poses.cpu().pin_memory()
    host = lambda t: t.numpy()
    r = mm.voxelize(host(spo_p), host(P_p), host(T_p), **cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        r = mm.voxelize(host(spo_p), host(P_p), host(T_p), **cfg)
    e2e_s = (time.perf_counter() - t0) / steps
    h2d = spo_p.numel() * 8 + P_p.numel() * 8 + T_p.numel() * 8
    d2h = sum(a.nbytes for a in r.values() if hasattr(a, "nbytes"))
    hbm, src = hbm_peak()
    # the level-1 sort runs ceil(bits / 8) passes over the packed keys
    span = _world_index_range(P_p.numpy(), spo_h, s.pose_init[:n_scans], cfg["voxel_size"])
    passes = -(-int(sum(int(x).bit_length() for x in span)) // 8)
    rl = {
        "cluster_pass": {"bound": "alu", "achieved": VOX_CLUSTER_FLOPS_PER_POINT * n_pts / (stage_ms["cluster_pass"] / 1e3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"},
        "keys": {"bound": "alu", "achieved": VOX_KEYS_FLOPS_PER_POINT * n_pts / (stage_ms["keys"] / 1e3) / 1e12,
                 "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"},
        "sort": {"bound": "hbm", "achieved": VOX_SORT_BYTES_PER_POINT(passes) * n_pts / (stage_ms["sort"] / 1e3) / 1e9,
                 "peak": hbm, "unit": "GB/s"},
    }
    for x in rl.values():
        x["frac"] = x["achieved"] / x["peak"]
    top = max(rl, key=lambda k: stage_ms[k])
    kname = {"cluster_pass": "l1_pieces", "keys": "l1_keys", "sort": "radix sort of the level-1 keys"}[top]
    tr = recorded_traffic(f"voxelize_{n_scans}", kname)
    roof = dict(rl[top], traffic=tr, kernel=kname,
                stage_ms=stage_ms[top], peak_source="FP64: 152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz"
                if rl[top]["bound"] == "alu" else src)
    # oracle on the first scans' points (bounded sample), scaled by points
    import oracle
    k = 1
    while k < n_scans and spo_h[k] < 25_000_000:
        k += 1
    Ph = P[: int(spo_h[k])].cpu().numpy()
    t0 = time.perf_counter()
    oracle.voxelize(spo_h[: k + 1], Ph, s.pose_init[:k], **cfg)
    cpu_s = time.perf_counter() - t0
    line = {
        "metric": "preprocessing points/s (L1 voxelisation, 3 levels, selection)", "workload": "voxelize",
        "value": n_pts / (ms / 1000.0), "unit": "points/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "points": n_pts, "voxels_out": int(v["level"].numel()),
        "obs_out": int(v["obs_scan"].numel()), "gpu_launches": int(launches), "clocks": clk,
        "e2e": {"value": n_pts / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1000.0,
                "scope": "ba_voxelize from pinned host points (adaptive loader: batches copied on a second "
                         "stream under the clustering) + ba_voxels_read to host",
                "loader_batches": int(r["batches"])},
        "roofline": roof,
        "stages_ms": {k2: round(x, 3) for k2, x in stage_ms.items()},
        "stage_rooflines": {k2: {"frac": round(x["frac"], 3), "bound": x["bound"]} for k2, x in rl.items()},
        "cpu_baseline": {"value": int(spo_h[k]) / cpu_s, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"points of the first {k} scans ({int(spo_h[k])} points)"},
        "config": {"workload": f"raw scans of the {n_scans}-scan scene ({n_pts} points) -> voxels",
                   "scans": n_scans, "voxel_size_m": cfg["voxel_size"], "levels": cfg["levels"],
                   "tau": cfg["tau"], "min_obs": cfg["min_obs"], "sort_passes": passes,
                   "inputs": "points resident on the device, larger than L2"},
    }
    del P, spo_p, P_p, r, v
    torch.cuda.empty_cache()
    return line


def _world_index_range(P, spo, poses, d):
    """Per axis, the span of the level-1 voxel indices (max - min), from the
    poses applied to each scan's points (host arithmetic, for the pass count)."""
    import numpy as np
    lo, hi = np.full(3, np.inf), np.full(3, -np.inf)
    for j in range(len(spo) - 1):
        Q = P[spo[j]:spo[j + 1]]
        if len(Q) == 0:
            continue
        W = Q @ poses[j, :9].reshape(3, 3).T + poses[j, 9:]
        lo, hi = np.minimum(lo, W.min(axis=0)), np.maximum(hi, W.max(axis=0))
    return np.floor(hi / d) - np.floor(lo / d)


def _line_fit(x, y):
    """Least-squares line y = a x + b and its R^2."""
    import numpy as np
    x, y = np.asarray(x, float), np.asarray(y, float)
    a, b = np.polyfit(x, y, 1)
    ss_res = float(((y - (a * x + b)) ** 2).sum())
    ss_tot = float(((y - y.mean()) ** 2).sum())
    return {"slope": float(a), "intercept": float(b), "r2": 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0}


def run_sweep(args):
    """The paper's scaling figure (Sec. V, Fig. 3) in shape: per-iteration
    evaluation time (voxel and scan passes, mixed path) against the number of
    clusters and the solver's time against the number of poses, on city
    scenes of 1/8 to full size; preprocessing time against the number of
    points on 1/8 to all of the 1,000-scan raw scans.  Each series gets a
    least-squares line and its R^2 (the paper reports linear growth)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2608_14266_gb300 as mm
    import scenegen
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    fracs = [0.125, 0.25, 0.5, 1.0]
    ev, sv = [], []
    for f in fracs:
        p = scenegen.config("city")
        side = math.sqrt(f)
        p = scenegen.replace(p, n_scans=int(p.n_scans * f), n_voxels=int(p.n_voxels * f),
                             box=(p.box[0] * side, p.box[1] * side, p.box[2]))
        scene = scenegen.make_scene(p)
        inputs = (torch.from_numpy(scene.voxel_off).to(dev), torch.from_numpy(scene.obs_scan).to(dev),
                  device_clusters_gpu(scene, torch, mm), torch.from_numpy(scene.pose_init).to(dev))
        res = measure(mm, torch, scene, inputs, mm.BA_MIXED, 300, 30, 30, lambda: None, 0)
        prof = res["prof"]
        per = {k: prof[k][0] / max(1, prof[k][1]) for k in ("voxel_pass", "scan_pass", "solve")}
        ev.append((scene.n_obs, per["voxel_pass"] + per["scan_pass"]))
        sv.append((scene.n_scans, per["solve"]))
        del inputs
        torch.cuda.empty_cache()
    # preprocessing: prefixes of the 1,000-scan raw scans
    s = scenegen.make_scene(scenegen.config("mid"))
    npo = s.params.pts_per_obs
    P = torch.empty((s.n_obs * npo, 3), dtype=torch.float64, device=dev)
    s.points_device(0, s.n_obs, P)
    order = torch.from_numpy(np.argsort(s.obs_scan, kind="stable")).to(dev)
    P = P.view(s.n_obs, npo, 3)[order].reshape(-1, 3).contiguous()
    spo_all = np.concatenate([[0], np.cumsum(np.bincount(s.obs_scan, minlength=s.n_scans) * npo)]).astype(np.int64)
    stream = torch.cuda.current_stream()
    pv = []
    for f in fracs:
        k = max(1, int(round(s.n_scans * f)))
        spo = torch.from_numpy(spo_all[: k + 1]).to(dev)
        n = int(spo_all[k])
        Pk, T = P[:n], torch.from_numpy(s.pose_init[:k]).to(dev)
        cfg = dict(voxel_size=0.5, levels=3, tau=0.1, min_obs=2, stream=stream, out="device")
        mm.voxelize(spo, Pk, T, **cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            mm.voxelize(spo, Pk, T, **cfg)
        e1.record(stream)
        torch.cuda.synchronize()
        pv.append((n, e0.elapsed_time(e1) / 3))
    line = {
        "metric": "scaling sweep (the paper's Fig. 3 in shape): times against problem size",
        "workload": "sweep", "n_gpus": 1, "higher_is_better": False, "dtype": "f32 (iterations) / f64 (preprocessing)",
        "data": "synthetic",
        "series": {
            "evaluation_ms_vs_clusters": {"points": ev, "fit": _line_fit(*zip(*ev))},
            "solve_ms_vs_poses": {"points": sv, "fit": _line_fit(*zip(*sv))},
            "preprocess_ms_vs_points": {"points": pv, "fit": _line_fit(*zip(*pv))},
        },
        "config": {"workload": "city scenes at 1/8, 1/4, 1/2 and full size (mixed path, 300 timed iterations "
                               "each); prefixes of the 1,000-scan raw scans (d = 0.5 m, 3 levels)"},
    }
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "voxelize":
        run_voxelize(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "batched":
        _standalone(batched_result, args)
    elif args.workload == "served":
        _standalone(served_result, args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

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
# (an FMA counts as 2): q = R m + t (18), q - a (3), R S R^T (45),
# N (q - a) (3), accumulation of M (48), sums of N (q - a) and N (4).
VOXEL_PASS_FLOP_PER_OBS = 121
# bytes one voxel-pass launch must move per observation slot: 10 doubles + a
# 4-byte scan index (the pose table and per-voxel outputs are small)
VOXEL_PASS_BYTES_PER_ELEM = 84
# mixed voxel pass: per observation 10 floats + a 4-byte scan index; per voxel
# the anchor and frame (12 floats), its length (4 B), the plane written (16 B)
MIXED_VOXEL_BYTES_PER_OBS = 44
MIXED_VOXEL_BYTES_PER_VOXEL = 68


def _args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000, help="timed LM iterations per rank")
    ap.add_argument("--warmup", type=int, default=30, help="untimed warm-up iterations")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["city", "mid", "tiny"], default="city")
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


def kernel_source_hash(kernel: str = "voxel_pass_f64") -> str:
    h = hashlib.sha256()
    main = "iter_mixed.cu" if "mixed" in kernel else "iter_f64.cu"
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


def time_oracle(scene, steps: int, warmup: int, total_budget_s: float):
    """Times oracle LM iterations on a bounded sample; returns the full-problem
    iterations per second and the description of the sample."""
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
    return frac / dt, dt, sample


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import scenegen
    scene = scenegen.make_scene(scene_params(scenegen, args, 0))
    budget = 150.0
    ips, dt, sample = time_oracle(scene, args.steps, args.warmup, budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": ips, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / ips, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene generator)",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "n_obs": scene.n_obs, "solver": "CPU oracle, FP64"},
        "plane_obs_per_s": ips * scene.n_obs,
        "e2e": {"value": ips, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": ips, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": sample},
    }
    print(json.dumps(line), flush=True)


def measure(mm, torch, scene, dev_inputs, precision, steps, warmup, S, barrier, local, profile=True):
    """Times `steps` LM iterations (solves of S iterations from the initial
    poses, state reset outside the timed region) with CUDA events on the
    library's stream; returns the timing, the kernel breakdown and clocks."""
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
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in reps]
    accepted = 0
    launches = 0
    acc0 = ba.stats()["accepted"]
    clocks = ClockSampler(_gpu_id(torch, local)) if profile else None
    if profile:
        time.sleep(0.3)
    ba.profile(profile)
    torch.cuda.nvtx.range_push("timed")
    t_wall0 = time.time()
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
    t_wall1 = time.time()
    torch.cuda.nvtx.range_pop()
    prof = ba.profile_read() if profile else None
    ba.profile(False)
    clk = clocks.stop(t_wall0, t_wall1) if clocks else None
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    ba.close()
    return {"ms": ms, "accepted": accepted, "launches": launches, "prof": prof, "clocks": clk}


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
    nbytes = MIXED_VOXEL_BYTES_PER_OBS * scene.n_obs + MIXED_VOXEL_BYTES_PER_VOXEL * scene.n_voxels
    achieved = nbytes / vp_avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(workload, "voxel_pass_mixed"), "kernel": "voxel_pass_mixed",
            "avg_launch_ms": vp_avg_s * 1000.0, "peak_source": src, "bytes_per_launch": nbytes}


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

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=torch.device("cuda", local))
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    scene = scenegen.make_scene(scene_params(scenegen, args, rank))
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
    e2e_times = []
    for _ in range(args.e2e_jobs):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mm.BundleAdjuster(cuda_stream=stream, precision=prec) as job:
            job.load_observations(scene.n_scans, vo_h.numpy(), os_h.numpy(), agg_h.numpy(), p0_h.numpy())
            job.iterate(S, stats=False)
            job.poses(out=out_h.numpy())
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = None
    if e2e_times:
        e2e_value = world * S * args.e2e_jobs / max_over_ranks(sum(e2e_times))
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
        ips, dt, sample = time_oracle(scene, 2, 1, args.cpu_seconds)
        cpu = {"value": ips, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": sample}
    per_obs = 44 if args.precision == "mixed" else 84
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded scene generator; points clustered on GPU)",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "n_scans": scene.n_scans,
                   "n_voxels": scene.n_voxels, "n_obs": scene.n_obs, "precision": args.precision,
                   "iters_per_solve": S, "accepted_iters": res["accepted"],
                   "l2": "inputs larger than L2 (per-pass clusters %.2f GB)" % (scene.n_obs * per_obs / 1e9),
                   "parallelism": f"{world} independent job(s), one per GPU"},
        "plane_obs_per_s": value * scene.n_obs,
        "fp64_path": fp64,
        "clocks": res["clocks"],
        "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": h2d / S, "d2h_bytes_per_step": d2h / S,
                "jobs": args.e2e_jobs, "scope": "ba_load_observations (pinned host clusters) + "
                                                f"{S} iterations + ba_poses to host, per job"},
        "gpu_launches": int(res["launches"]),
        "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items()},
        "roofline": roofline,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

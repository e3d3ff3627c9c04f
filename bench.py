#!/usr/bin/env python
"""Throughput of camera covariance propagation on one GB300 (or N replicas).

A step is one pass of the whole path on one scene: ccov_information ->
ccov_schur -> ccov_nullspace -> ccov_covariance (steps (a)-(d)).  The
workload is the synthetic 4000-camera shell scene (400k points, track length
1 + Geometric(1/7), about 3.2M observations, reduced camera matrix
36000 x 36000).  For the mixed form the line also carries one pass of the
plain FP64 GPU form on the same scene (`vs_fp64_gpu`: its time and the mixed
blocks' relative Frobenius error against it), and a short timing of the
batched form below (`batch256`; `--no-batch-extra` leaves it out).  `value` =
cameras / s with the inputs resident on the device;
`e2e` = the same through the C ABI with host buffers (host-to-device upload and
the device-to-host copy of the 9x9 blocks inside every timed step).

`--workload surrogate` trains the learned surrogate on exact blocks of
2000 scenes (n ~ U{50..500}) and times its prediction on the 4000-camera
scene (value = cameras / s of ccov_information + features + the nullspace
rows + the gauge term of the base + prediction).

`--workload batch256` times the batched form instead: 256 independent
sub-reconstructions (n ~ U{10..300} cameras, 100 points per camera, track
length 1 + Geometric(0.2)), all four steps of every scene as grouped launches
(one per step for all scenes) recorded once as a CUDA graph and replayed, one
replay per step; `value` = cameras / s over the whole batch.

`--workload subrecon` times the Sec. 5 pipeline on a 1000-camera scene with
visibility locality (sub-reconstructions of 100 view-graph neighbours, three
decompositions, minimum-trace merge), with the error against the full scene.

`--workload update` times the covariance update after 200 added observations
(Sec. 5, Woodbury) on the 4000-camera scene, against a new step (d) of the
merged scene, and the update's time for 20, 50 and 800 added observations.

`--workload shell1k` (or any scene name of synth.workload) runs the default
step on that scene.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead, on a bounded sub-scene of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "camera covariances/s (4k-cam scene), mixed vs FP64 GPU at ≤1e-6 rel error"
UNIT = "camera covariances/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (vector and tensor), nominal


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="shell4k")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--cpu-sample-cams", type=int, default=900)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--no-batch-extra", action="store_true",
                    help="leave the batched form's figure out of the default (4000-camera) line")
    ap.add_argument("--e2e-steps", type=int, default=0, help="0: the same as --steps")
    ap.add_argument("--surr-scenes", type=int, default=2000)
    ap.add_argument("--surr-epochs", type=int, default=30)
    ap.add_argument("--surr-batch", type=int, default=4096)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel_tag: str, flops_per_launch: float):
    """DRAM bytes per launch from the committed ncu capture (bytes per executed
    flop there, times this run's flops per launch: the result tile traffic grows
    with the tiles, as the flops do), if the kernel source has not changed since
    the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_tag)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != rec["source_sha"]:
        return None
    return rec["dram_bytes_per_flop"] * flops_per_launch


def block_errors(S, R, cams=None):
    """Per-block error measures of S against R ((n, 9, 9) arrays): relative
    Frobenius of the block, of the block scaled by diag(R)^-1/2, of its 6x6
    pose and 3x3 intrinsic sub-blocks, and (with `cams`) the paper's err
    (Sec. 6: mean over the entries of sqrt(|S - R|) / O, O = sqrt(E|P| E|P|^T))."""
    import numpy as np

    def fro(a, b):
        return np.linalg.norm(a - b, axis=(-2, -1)) / np.linalg.norm(b, axis=(-2, -1))

    d = 1.0 / np.sqrt(np.abs(np.einsum("...ii->...i", R)))
    Dd = d[..., :, None] * d[..., None, :]
    out = {"rel_fro": fro(S, R), "norm_err": fro(S * Dd, R * Dd), "pose_err": fro(S[:, :6, :6], R[:, :6, :6]),
           "intr_err": fro(S[:, 6:, 6:], R[:, 6:, 6:])}
    if cams is not None:
        e = np.abs(cams).mean(axis=0)
        out["paper_err"] = (np.sqrt(np.abs(S - R)) / np.sqrt(np.outer(e, e))).mean(axis=(-2, -1))
    return out


def dist_init(n_gpus: int):
    import torch
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", 0))
    return 0, 1, 0


def barrier_max(x: float, world: int):
    """Maximum of x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_sample(scene, k: int):
    """The oracle as it stands on a k-camera sub-scene (a bounded sample)."""
    import numpy as np

    from oracle import covariance
    from paper_1808_02414_gb300 import synth

    sub = synth.subscene(scene, np.arange(min(k, scene.n)))
    t0 = time.perf_counter()
    covariance.camera_covariance(sub)
    dt = time.perf_counter() - t0
    return sub, dt


def run_reference(args):
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return
    if args.workload == "batch256":
        run_reference_batch(args)
        return
    from paper_1808_02414_gb300 import synth
    # the surrogate's and the update's reference is the exact method on the
    # scene they run on (for the update: the covariance from scratch); that of
    # the sub-reconstructions, the exact method on their scene
    if args.workload in ("surrogate", "update"):
        scene = synth.workload("shell4k")
    elif args.workload == "subrecon":
        scene = synth.local_scene(n=1000, m=100_000, seed=3)
    else:
        scene = synth.workload(args.workload)
    times = []
    sub = None
    for i in range(args.warmup + args.steps):
        sub, dt = cpu_oracle_sample(scene, args.cpu_sample_cams)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = sub.n / (ms / 1e3)
    cores = os.cpu_count()
    sample = (f"{sub.n}-camera sub-scene ({sub.m} points, {sub.t} observations) of the "
              f"{args.workload} workload, full oracle route (bordered Schur + LU), per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cameras": scene.n, "points": scene.m,
                       "observations": scene.t, "sample_cameras": sub.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    """The oracle on whole scenes of the batch (about 12 s per step)."""
    scenes = batch_workload()
    times, sample = [], None
    for i in range(args.warmup + args.steps):
        cams, used, dt = cpu_oracle_batch_sample(scenes)
        if i >= args.warmup:
            times.append(cams / dt)
        sample = f"the first {used} scenes of the batch ({cams} cameras) per step"
    value = statistics.mean(times)
    line = {"impl": "reference", "metric": "camera covariances/s (batched sub-reconstructions)", "value": value,
            "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cams / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch256", "scenes": len(scenes), "cameras": sum(sc.n for sc in scenes)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov, synth

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene = synth.workload(args.workload)
    prec = ccov.CCOV_PREC_MIXED if args.precision == "mixed" else ccov.CCOV_PREC_FP64
    stream = torch.cuda.current_stream(dev)

    # inputs resident in HBM
    cams = torch.from_numpy(scene.cams).to(dev)
    pts = torch.from_numpy(scene.pts).to(dev)
    rec = scene.obs_records()
    obs = torch.from_numpy(rec.view(np.uint8)).to(dev)
    out = torch.empty((scene.n, 9, 9), dtype=torch.float64, device=dev)
    # the timed context records no per-GEMM events; a second, profiled
    # context gives the GEMM statistics from one separate step
    ctx = ccov.Context(cams, pts, obs, scene.sigma, precision=prec, stream=stream.cuda_stream)

    def step(c=ctx):
        c.ccov_information()
        c.ccov_schur()
        c.ccov_nullspace()
        c.ccov_covariance(out=out)
        return c.ccov_get_stats()

    for _ in range(args.warmup):
        step()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        stats.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_total = barrier_max(e0.elapsed_time(e1), world)
    ms_step = ms_total / args.steps
    value = scene.n * args.steps * world / (ms_total / 1e3)

    # end to end through the C ABI with host buffers (pinned)
    h_cams = torch.from_numpy(scene.cams).pin_memory()
    h_pts = torch.from_numpy(scene.pts).pin_memory()
    h_obs = torch.from_numpy(rec.view(np.uint8)).pin_memory()
    h_out = torch.empty((scene.n, 9, 9), dtype=torch.float64).pin_memory()
    ctx_h = ccov.Context(scene.cams, scene.pts, rec, scene.sigma, precision=prec,
                         stream=stream.cuda_stream)
    h2d = scene.cams.nbytes + scene.pts.nbytes + rec.nbytes
    d2h = scene.n * 81 * 8
    np_cams, np_pts = h_cams.numpy(), h_pts.numpy()
    np_obs = h_obs.numpy().view(rec.dtype)
    np_out = h_out.numpy()
    barrier(world)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = args.e2e_steps or args.steps
    f0.record(stream)
    for _ in range(e2e_steps):
        ctx_h.ccov_load(np_cams, np_pts, np_obs)
        ctx_h.ccov_information()
        ctx_h.ccov_schur()
        ctx_h.ccov_nullspace()
        ccov.load().ccov_covariance(ctx_h._h, np_out.ctypes.data, ccov.CCOV_MEM_HOST, None)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = barrier_max(f0.elapsed_time(f1), world) / e2e_steps
    e2e_value = scene.n * world / (ms_e2e / 1e3)
    ctx_h.close()

    # GEMM statistics: one step of a profiled context (events around every
    # trailing-update GEMM), outside the timed region
    ctx_p = ccov.Context(cams, pts, obs, scene.sigma, precision=prec, stream=stream.cuda_stream, profile=True)
    pstats = [step(ctx_p)]
    ctx_p.close()

    # roofline of the dominant kernel family: the trailing-update GEMMs of step (d)
    # roofline of the dominant kernel family, the trailing-update GEMMs of
    # step (d): achieved = the method's algorithmic work (2/3) N^3 (Cholesky
    # N^3/3 + triangular inverse N^3/3, N = 9n) / the GEMMs' summed event time
    pk, src = peaks()
    gemm_ms = statistics.mean(s["ms_gemm"] for s in pstats)
    exec_flops = statistics.mean(s["gemm_flops"] for s in pstats)
    gemm_launches = int(statistics.mean(s["gemm_launches"] for s in pstats))
    N = 9 * scene.n
    alg_flops = 2.0 / 3.0 * float(N) ** 3
    achieved = alg_flops / (gemm_ms / 1e3) / 1e12
    work = f"(2/3) N^3 = {alg_flops:.3e} flop per step, N = {N}"
    if prec == ccov.CCOV_PREC_FP64:
        peak = FP64_NOMINAL_GFLOPS / 1e3
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for("gemm64", exec_flops / max(gemm_launches, 1)),
                "kernel": "gemm64_kernel (FP64 trailing updates)", "peak_source": "nominal FP64",
                "work": work, "launches_per_step": gemm_launches, "ms_per_step": gemm_ms,
                "share_of_step": gemm_ms / ms_step}
        dtype = "f64"
    else:
        peak = pk["bf16_tflops_sustained"]
        ex_tf = exec_flops / (gemm_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for("ozaki_gemm", exec_flops / max(gemm_launches, 1)),
                "kernel": "ozaki_gemm (split-bf16 tcgen05 trailing updates)",
                "peak_source": f"bf16 sustained ({src})", "work": work,
                "executed": {"flops_per_step": exec_flops, "tflops": ex_tf, "frac": ex_tf / peak,
                             "what": "every kept 128x64 tile x s(s+1)/2 digit products"},
                "launches_per_step": gemm_launches, "ms_per_step": gemm_ms, "share_of_step": gemm_ms / ms_step,
                "timing": "separate profiled step; events around each GEMM launch, which overlap kernels "
                          "of the other stream (Cholesky and inverse run concurrently)"}
        dtype = "bf16"
    last = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "cameras": scene.n, "points": scene.m,
                       "observations": scene.t, "N": 9 * scene.n, "precision": args.precision,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set > L2: the dense reduced matrix alone is "
                             f"{(9 * scene.n) ** 2 * 8 / 1e9:.1f} GB"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "roofline": roof,
            "phases_ms": {k: last[k] for k in ("ms_information", "ms_schur", "ms_nullspace",
                                                "ms_covariance", "ms_factor", "ms_inverse")}}
    ctx.close()
    if prec == ccov.CCOV_PREC_MIXED and not args.no_fp64_check:
        # the same scene through the plain FP64 GPU form, once: its time and the
        # mixed form's per-block error against it
        mixed = out.cpu().numpy()
        ref = torch.empty_like(out)
        with ccov.Context(cams, pts, obs, scene.sigma, precision=ccov.CCOV_PREC_FP64,
                          stream=stream.cuda_stream) as c64:
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            c64.run(out=ref)
            g1.record(stream)
            torch.cuda.synchronize()
            ms64 = g0.elapsed_time(g1)
        ref = ref.cpu().numpy()
        errs = block_errors(mixed, ref)
        line["vs_fp64_gpu"] = {"ms_per_step": ms64, "value": scene.n / (ms64 / 1e3), "unit": UNIT,
                               "speedup_of_mixed": ms64 / ms_step,
                               "max_rel_fro_per_block": float(errs["rel_fro"].max()),
                               "median_rel_fro_per_block": float(np.median(errs["rel_fro"])),
                               "max_norm_err_per_block": float(errs["norm_err"].max()),
                               "max_pose_err_per_block": float(errs["pose_err"].max()),
                               "max_intr_err_per_block": float(errs["intr_err"].max())}
    if (world == 1 and args.workload == "shell4k" and prec == ccov.CCOV_PREC_MIXED
            and not args.no_batch_extra):
        line["batch256"] = batch_extra(dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sub, dt = cpu_oracle_sample(scene, args.cpu_sample_cams)
        line["cpu_baseline"] = {"value": sub.n / dt, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{sub.n}-camera sub-scene ({sub.m} points, {sub.t} "
                                          f"observations) of {args.workload}, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


BATCH_K = 256


def batch_extra(dev, stream, warmup: int = 3, steps: int = 5):
    """The batched form (`--workload batch256`: 256 scenes of 10-300 cameras,
    mixed, grouped launches replayed as one graph) timed briefly, so that the
    default line carries its figure too: device-resident inputs, CUDA events
    around `steps` replays after `warmup`."""
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov
    scenes = batch_workload()
    ctxs, outs = [], []
    for sc in scenes:
        rec = sc.obs_records()
        ctxs.append(ccov.Context(torch.from_numpy(sc.cams).to(dev), torch.from_numpy(sc.pts).to(dev),
                                 torch.from_numpy(rec.view(np.uint8)).to(dev), sc.sigma,
                                 precision=ccov.CCOV_PREC_MIXED))
        outs.append(torch.empty((sc.n, 9, 9), dtype=torch.float64, device=dev))
    try:
        with ccov.Batch(ctxs, outs) as b:
            info = b.info()
            for _ in range(warmup):
                b.run(stream.cuda_stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                b.run(stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
    finally:
        for c in ctxs:
            c.close()
    ms = e0.elapsed_time(e1) / steps
    cams = sum(sc.n for sc in scenes)
    return {"value": cams / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "scenes": len(scenes), "cameras": cams, "launches_per_step": int(info["launches"]),
            "form": "grouped launches, one CUDA graph replay per step (bench.py --workload batch256)"}


def batch_workload():
    from paper_1808_02414_gb300 import synth
    return synth.batch_scenes(k=BATCH_K, n_lo=10, n_hi=300, pts_per_cam=100, p_geom=0.2)


def cpu_oracle_batch_sample(scenes, budget_s: float = 12.0):
    """The oracle as it stands on whole scenes of the batch, in batch order,
    until about `budget_s` seconds of CPU work (a bounded sample)."""
    from oracle import covariance
    cams, t0 = 0, time.perf_counter()
    used = 0
    for sc in scenes:
        covariance.camera_covariance(sc)
        cams += sc.n
        used += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return cams, used, time.perf_counter() - t0


def run_batch(args):
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scenes = batch_workload()
    prec = ccov.CCOV_PREC_MIXED if args.precision == "mixed" else ccov.CCOV_PREC_FP64
    stream = torch.cuda.current_stream(dev)
    cams_total = sum(sc.n for sc in scenes)

    # inputs resident in HBM; one context (and stream) per scene
    ctxs, outs = [], []
    for sc in scenes:
        rec = sc.obs_records()
        ctxs.append(ccov.Context(torch.from_numpy(sc.cams).to(dev), torch.from_numpy(sc.pts).to(dev),
                                 torch.from_numpy(rec.view(np.uint8)).to(dev), sc.sigma,
                                 precision=prec))
        outs.append(torch.empty((sc.n, 9, 9), dtype=torch.float64, device=dev))
    batch = ccov.Batch(ctxs, outs)
    info = batch.info()
    for _ in range(args.warmup):
        batch.run(stream.cuda_stream)
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.run(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_total = barrier_max(e0.elapsed_time(e1), world)
    ms_step = ms_total / args.steps
    value = cams_total * args.steps * world / (ms_total / 1e3)
    batch.close()

    # the per-scene form of the same batch (each scene's own kernels on its own
    # stream, one graph), and the direct calls without a graph
    with ccov.Batch(ctxs, outs, form=ccov.CCOV_BATCH_PER_SCENE) as bp:
        bp.run(stream.cuda_stream)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        bp.run(stream.cuda_stream)
        p1.record(stream)
        torch.cuda.synchronize()
        ms_per_scene_graph = p0.elapsed_time(p1)
        per_scene_launches = bp.info()["launches"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ccov.ccov_batch_covariance(ctxs, outs)
    ms_direct = 1e3 * (time.perf_counter() - t0)
    for c in ctxs:
        c.close()

    # roofline: the batch's algorithmic work sum (2/3) N_b^3 (Cholesky and
    # triangular inverse of every scene) over the whole step time, a lower
    # bound of the GEMMs' own rate (the step also holds steps (a)-(c), the
    # diagonal blocks and the slicing)
    pk, src = peaks()
    alg = sum(2.0 / 3.0 * float(9 * sc.n) ** 3 for sc in scenes)
    achieved = alg / (ms_step / 1e3) / 1e12
    if prec == ccov.CCOV_PREC_FP64:
        peak, bound, dtype, kern, psrc = FP64_NOMINAL_GFLOPS / 1e3, "alu", "f64", "gemm64_kernel", "nominal FP64"
    else:
        peak, bound, dtype = pk["bf16_tflops_sustained"], "tensor", "bf16"
        kern, psrc = "ozaki_gemm (grouped split-bf16 tcgen05 trailing updates)", f"bf16 sustained ({src})"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kern, "peak_source": psrc,
            "work": f"sum over scenes of (2/3) N_b^3 = {alg:.3e} flop per step",
            "note": "work / whole step time (a lower bound of the dominant kernel's rate)"}

    # end to end through the same grouped batch: every step loads each
    # scene's pinned host inputs into its context, replays the batch and
    # copies every block back to pinned host memory
    pinned, e2e_ctx = [], []
    for sc in scenes:
        rec = sc.obs_records()
        hc = torch.from_numpy(sc.cams).pin_memory()
        hp = torch.from_numpy(sc.pts).pin_memory()
        ho = torch.from_numpy(rec.view(np.uint8)).pin_memory()
        pinned.append((hc.numpy(), hp.numpy(), ho.numpy().view(rec.dtype)))
        e2e_ctx.append(ccov.Context(sc.cams, sc.pts, rec, sc.sigma, precision=prec))
    d_outs = [torch.empty((sc.n, 9, 9), dtype=torch.float64, device=dev) for sc in scenes]
    h_outs = [torch.empty((sc.n, 9, 9), dtype=torch.float64).pin_memory() for sc in scenes]
    h2d = sum(sc.cams.nbytes + sc.pts.nbytes + sc.t * 24 for sc in scenes)
    d2h = cams_total * 81 * 8
    e2e_steps = args.e2e_steps or args.steps
    with ccov.Batch(e2e_ctx, d_outs) as be:
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(e2e_steps):
            for c, (a, b, o) in zip(e2e_ctx, pinned):
                c.ccov_load(a, b, o)
            be.run(stream.cuda_stream)
            for h, d in zip(h_outs, d_outs):
                h.copy_(d, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
    ms_e2e = barrier_max(f0.elapsed_time(f1), world) / e2e_steps
    for c in e2e_ctx:
        c.close()

    line = {"metric": "camera covariances/s (batched sub-reconstructions)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": "batch256", "scenes": len(scenes), "cameras": cams_total,
                       "points": sum(sc.m for sc in scenes), "observations": sum(sc.t for sc in scenes),
                       "precision": args.precision,
                       "form": "grouped launches (one per step for all scenes), one CUDA graph replay per step"
                               if info["form"] == ccov.CCOV_BATCH_GROUPED else "per-scene kernels, one CUDA graph",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set > L2: the reduced matrices total "
                             f"{sum((9 * sc.n) ** 2 for sc in scenes) * 8 / 1e9:.1f} GB"},
            "clocks": clk,
            "e2e": {"value": cams_total * world / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
            "gpu_launches": int(info["launches"]) * args.steps,
            "roofline": roof,
            "batch_form": {"launches_per_step": int(info["launches"]),
                           "autotuned_gemm": {"ctas": info["gemm_ctas"], "stages": info["gemm_stages"],
                                              "tune_ms": info["tune_ms"]},
                           "per_scene_graph": {"ms_per_step": ms_per_scene_graph,
                                               "launches_per_step": int(per_scene_launches)},
                           "direct_batched_call_ms": ms_direct}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cams, used, dt = cpu_oracle_batch_sample(scenes)
        line["cpu_baseline"] = {"value": cams / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"the first {used} scenes of the batch ({cams} cameras), {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# kernels of one surrogate step: cam_prep, obs_info, point_ainv, cam_info
# (ccov_information); features, centre spread, centre feature; nullspace rows;
# gauge sums, L_c, gauge rows; base factor; pack, 4 GEMMs, output (prediction)
SURR_STEP_LAUNCHES = 18


def _training_scene(spec):
    from paper_1808_02414_gb300 import synth
    return synth.training_scene(spec)


def surrogate_training_set(n_scenes: int, n_heldout: int = 30, group: int = 32):
    """Per camera of the training scenes, on the device: features, L_z, gauge
    rows Q and the exact blocks; the same for `n_heldout` further scenes of
    the same distribution.  Scenes are drawn in worker processes (spawned, so
    that no worker inherits a CUDA context) and solved exactly with the FP64
    path in batches of `group` contexts."""
    import multiprocessing as mp

    import torch

    from paper_1808_02414_gb300 import ccov, surrogate, synth

    specs = synth.training_scene_specs(n_scenes + n_heldout)
    train, held = [], []
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        pending, seen = [], 0
        for sc in pool.imap(_training_scene, specs, chunksize=4):
            pending.append(sc)
            seen += 1
            if len(pending) < group and seen not in (n_scenes, len(specs)):
                continue
            _solve_group(pending, train if seen <= n_scenes else held, ccov, surrogate, torch)
            pending = []

    def cat(parts):
        return tuple(torch.cat(a) for a in zip(*parts)) if parts else None

    return cat(train), cat(held)


def _solve_group(scenes, out, ccov, surrogate, torch):
    ctxs = [ccov.from_scene(sc) for sc in scenes]
    outs = [torch.empty((sc.n, 9, 9), dtype=torch.float64, device="cuda") for sc in scenes]
    try:
        ccov.ccov_batch_covariance(ctxs, outs)
        for c, o in zip(ctxs, outs):
            f, lz = surrogate.features(c)
            out.append((f, lz, surrogate.gauge_rows(c, lz), o))
    finally:
        for c in ctxs:
            c.close()


def _gaussian_kl(pred, true):
    """KL(N(0, true) || N(0, pred)) per 9x9 block (unit-free error measure)."""
    import numpy as np
    Pi = np.linalg.inv(pred)
    return 0.5 * (np.einsum("iab,iba->i", Pi, true) - true.shape[1] + np.linalg.slogdet(pred)[1]
                  - np.linalg.slogdet(true)[1])


def _cov_from_target(t, Lz):
    """Sigma = L_z^-T L L^T L_z^-1 for network outputs t in the Cholesky
    target form (9 log-diagonal entries, then the strict lower triangle row
    by row), as the surrogate decodes them."""
    import numpy as np
    n = t.shape[0]
    L = np.zeros((n, 9, 9))
    k = np.arange(9)
    L[:, k, k] = np.exp(t[:, :9])
    il = np.tril_indices(9, -1)
    L[:, il[0], il[1]] = t[:, 9:]
    Li = np.linalg.inv(Lz)
    return Li.transpose(0, 2, 1) @ (L @ L.transpose(0, 2, 1)) @ Li


def _surrogate_accuracy(sm, f, lz, q, truth):
    """Median and p90 Gaussian KL against the exact blocks of the network's
    prediction, of the base with the fitted gauge term alone, of Z_ii^-1 and
    of a constant correction around the base."""
    import numpy as np
    T = sm.apply_gauge(lz, q)
    pred = sm.predict(f, T).cpu().numpy()
    Tn, L = T.cpu().numpy(), lz.cpu().numpy()
    mu_t = sm.normalization()[128:173].astype(np.float64)
    n = L.shape[0]
    zero = np.zeros((n, 45))
    f48 = f[:, 48].cpu().numpy().astype(np.float64)
    hs = np.where(f48 > 0, f48, 1.0)[:, None]        # the output head's size scale
    kl = {"surrogate": _gaussian_kl(pred, truth),
          "gauge_base": _gaussian_kl(_cov_from_target(zero, Tn), truth),
          "local_block_inverse": _gaussian_kl(_cov_from_target(zero, L), truth),
          "constant_correction": _gaussian_kl(_cov_from_target(hs * mu_t, Tn), truth)}
    out = {k: {"median_kl": float(np.median(v)), "p90_kl": float(np.percentile(v, 90))} for k, v in kl.items()}
    out["surrogate"]["median_rel_fro"] = float(np.median(
        np.linalg.norm(pred - truth, axis=(1, 2)) / np.linalg.norm(truth, axis=(1, 2))))
    out["cameras"] = int(n)
    return out


def run_surrogate(args):
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov, surrogate, synth

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    t0 = time.perf_counter()
    (F, LZ, QG, SG), held = surrogate_training_set(args.surr_scenes)
    data_s = time.perf_counter() - t0
    N, B = int(F.shape[0]), args.surr_batch
    steps = max(1, args.surr_epochs * N // B)
    idx = torch.from_numpy(synth.minibatch_indices(N, B, steps, seed=11)).to(dev)
    sm = surrogate.Surrogate(synth.surrogate_init(0), max_batch=B, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sm.fit_gauge(LZ, QG, SG)
    e1.record(stream)
    torch.cuda.synchronize()
    gauge_fit_ms = e0.elapsed_time(e1)
    TG = surrogate.targets(sm.apply_gauge(LZ, QG), SG)
    del LZ, QG, SG
    sm.fit_normalization(F, TG)
    torch.cuda.synchronize()
    e0.record(stream)
    losses = sm.train(F, TG, idx, 1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    ms_train_step = train_ms / steps
    accuracy = {"heldout_scenes_50_500_cams": _surrogate_accuracy(sm, *held[:3], held[3].cpu().numpy())}

    # evaluation on the 4000-camera scene: exact blocks from the mixed path
    scene = synth.workload("shell4k")
    cams = torch.from_numpy(scene.cams).to(dev)
    pts = torch.from_numpy(scene.pts).to(dev)
    rec = scene.obs_records()
    obs = torch.from_numpy(rec.view(np.uint8)).to(dev)
    exact = torch.empty((scene.n, 9, 9), dtype=torch.float64, device=dev)
    with ccov.Context(cams, pts, obs, scene.sigma, precision=ccov.CCOV_PREC_MIXED, stream=stream.cuda_stream) as cx:
        cx.run(out=exact)
    ctx = ccov.Context(cams, pts, obs, scene.sigma, stream=stream.cuda_stream)

    def step():
        ctx.ccov_information()
        f, lz = surrogate.features(ctx)
        ctx.ccov_nullspace()
        q = surrogate.gauge_rows(ctx, lz)
        return sm.predict(f, sm.apply_gauge(lz, q)), f, lz, q

    for _ in range(args.warmup):
        pred, f, lz, q = step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        pred, f, lz, q = step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = barrier_max(e0.elapsed_time(e1), world) / args.steps
    value = scene.n * world / (ms_step / 1e3)

    # end to end with host buffers: upload, the three calls, the blocks back
    hc = torch.from_numpy(scene.cams).pin_memory().numpy()
    hp = torch.from_numpy(scene.pts).pin_memory().numpy()
    ho = torch.from_numpy(rec.view(np.uint8)).pin_memory().numpy().view(rec.dtype)
    hout = torch.empty((scene.n, 9, 9), dtype=torch.float64).pin_memory()
    ctx_h = ccov.Context(scene.cams, scene.pts, rec, scene.sigma, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx_h.ccov_load(hc, hp, ho)
    ctx_h.ccov_information()
    f2, l2 = surrogate.features(ctx_h)
    ctx_h.ccov_nullspace()
    hout.copy_(sm.predict(f2, sm.apply_gauge(l2, surrogate.gauge_rows(ctx_h, l2))))
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    ctx_h.close()

    accuracy["shell4k_4000_cams"] = _surrogate_accuracy(sm, f, lz, q, exact.cpu().numpy())
    ctx.close()

    # executed tensor flops of one training step (padded widths 128/256/256/256/128)
    Bp = (B + 127) // 128 * 128
    fwd = 2.0 * Bp * (128 * 256 + 2 * 256 * 256 + 256 * 128)
    flops_step = fwd + (2.0 * Bp * (128 * 256 + 2 * 256 * 256)) + fwd
    pk, src = peaks()
    achieved = flops_step / (ms_train_step / 1e3) / 1e12
    line = {"metric": "camera covariances/s (surrogate, 4k-cam scene)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "surrogate", "train_scenes": args.surr_scenes, "train_samples": N,
                       "batch": B, "train_steps": steps, "eval": "shell4k (4000 cameras)",
                       "step": "ccov_information + surrogate features + ccov_nullspace + gauge rows "
                               "+ base factor + prediction",
                       "l2": "eval inputs 90 MB + blocks, working set > L2 in the information step"},
            "clocks": clk,
            "e2e": {"value": scene.n / (ms_e2e / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": scene.cams.nbytes + scene.pts.nbytes + rec.nbytes,
                    "d2h_bytes_per_step": scene.n * 81 * 8, "ms_per_step": ms_e2e},
            "gpu_launches": SURR_STEP_LAUNCHES * args.steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / pk["bf16_tflops"], "traffic": None,
                         "kernel": "mlp_gemm (training step, 11 GEMMs + pack/loss/Adam, one graph node each)",
                         "peak_source": f"bf16 burst ({src})",
                         "note": "executed GEMM flops per training step / whole step time: launch-bound"},
            "training": {"data_seconds": data_s, "gauge_fit_ms": gauge_fit_ms, "ms_per_step": ms_train_step,
                         "samples_per_s": B / (ms_train_step / 1e3), "loss_first": float(losses[:10].mean()),
                         "loss_last": float(losses[-50:].mean())},
            "accuracy_vs_exact": accuracy}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import nullspace as NS, surrogate as S
        sub = synth.subscene(scene, np.arange(300))
        t0 = time.perf_counter()
        f_o, lz_o = S.features(sub)
        q_o = S.gauge_rows(lz_o, NS.camera_rows_closed_form(sub).reshape(sub.n, 9, 7))
        norm = sm.normalization().astype(np.float64)
        S.predict(S.unpack(sm.params().astype(np.float64)), f_o, S.base_factor(lz_o, q_o, sm.gauge()),
                  (norm[:64], norm[64:128], norm[128:173], norm[173:]))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sub.n / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"features + prediction of a {sub.n}-camera sub-scene, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_subrecon(args):
    """Sec. 5 pipeline on a 1000-camera scene with visibility locality: the
    cameras' covariances from sub-reconstructions of k = 100 view-graph
    neighbours, three decompositions, minimum-trace merge; error against the
    full scene's covariances (mixed form)."""
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov, synth

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    scene = synth.local_scene(n=1000, m=100_000, seed=3)
    k, D = 100, 3
    orders = synth.decomposition_orders(scene.n, D, seed=7)
    for _ in range(args.warmup):
        ccov.subrecon_covariances(scene, k, orders)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out, cover, nsub = ccov.subrecon_covariances(scene, k, orders)
    torch.cuda.synchronize()
    ms_step = barrier_max(1e3 * (time.perf_counter() - t0), world) / args.steps
    clk = clocks.stop()
    full = ccov.camera_covariances(scene, precision=ccov.CCOV_PREC_MIXED)
    errs = block_errors(out, full, scene.cams)
    value = scene.n * world / (ms_step / 1e3)
    line = {"metric": "camera covariances/s (sub-reconstructions of a 1000-camera scene)", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "subrecon", "cameras": scene.n, "points": scene.m, "observations": scene.t,
                       "cams_per_sub": k, "decompositions": D, "sub_reconstructions": int(nsub),
                       "step": "ccov_subrecon_covariance from host inputs: plan, extraction, contexts, "
                               "grouped batch, merge (host clock around the call)"},
            "clocks": clk,
            "e2e": {"value": value, "unit": UNIT,
                    "h2d_bytes_per_step": scene.cams.nbytes + scene.pts.nbytes + scene.t * 24,
                    "d2h_bytes_per_step": scene.n * 81 * 8, "ms_per_step": ms_step},
            "gpu_launches": None,
            "error_vs_full_scene": {k2: {"median": float(np.median(v)), "mean": float(np.mean(v)),
                                         "p90": float(np.percentile(v, 90))} for k2, v in errs.items()},
            "cover": {"min": int(cover.min()), "mean": float(cover.mean())}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_update(args):
    """Covariance after adding observations (Sec. 5, Woodbury): the 4000-camera
    scene's factorisation from one step (d), then `UPDATE_K` added observations
    (20 on each of UPDATE_K / 20 cameras) per step through
    ccov_update_observations; checked against a new step (d) of the merged
    scene on the GPU (same precision), whose time is reported beside it."""
    import numpy as np
    import torch

    from paper_1808_02414_gb300 import ccov, synth

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prec = ccov.CCOV_PREC_MIXED if args.precision == "mixed" else ccov.CCOV_PREC_FP64
    scene = synth.workload("shell4k")
    k = UPDATE_K
    merged, added = synth.added_observations(scene, k, cams=np.arange(0, scene.n, scene.n // (k // 20))[: k // 20],
                                             seed=21)
    add = added.obs_records()
    out = torch.empty((scene.n, 9, 9), dtype=torch.float64, device=dev)
    ctx = ccov.from_scene(scene, precision=prec, stream=stream.cuda_stream)
    ctx.run(out=out)
    for _ in range(args.warmup):
        ctx.ccov_update_observations(add, out=out)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        ctx.ccov_update_observations(add, out=out)
        launches += ctx.ccov_get_stats()["update_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = barrier_max(e0.elapsed_time(e1), world) / args.steps
    upd = out.cpu().numpy()
    # end to end: host records in, host blocks out
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host = ctx.ccov_update_observations(add)
    ms_e2e = barrier_max(1e3 * (time.perf_counter() - t0), world) / args.steps
    assert np.array_equal(host, upd)
    # the same result by a new step (d) of the merged scene
    with ccov.from_scene(merged, precision=prec, stream=stream.cuda_stream) as c2:
        ref = torch.empty_like(out)
        c2.run(out=ref)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        c2.run(out=ref)
        g1.record(stream)
        torch.cuda.synchronize()
        ms_full = g0.elapsed_time(g1)
    errs = block_errors(upd, ref.cpu().numpy())
    # the time for other numbers of added observations (same scene, one context)
    by_k = {}
    for kk in UPDATE_K_SWEEP:
        _, add_k = synth.added_observations(scene, kk, seed=22)
        rec_k = add_k.obs_records()
        ctx.ccov_update_observations(rec_k, out=out)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(2):
            ctx.ccov_update_observations(rec_k, out=out)
        h1.record(stream)
        torch.cuda.synchronize()
        by_k[str(kk)] = h0.elapsed_time(h1) / 2
    ctx.close()
    value = scene.n * world / (ms_step / 1e3)
    # roofline of the tensor-core products of one update: the algorithmic work
    # (X V and X^T W, N^2 r flop each with X triangular; W^T W and Y X_S^T, N r^2
    # each, r = 2k) and the executed digit products (every 128 x 64 tile of
    # the K = 256 panel GEMMs x 15 products for S = 5), both over the whole
    # update time (a lower bound of the GEMMs' rate)
    N, r = 9 * scene.n, 2 * k
    Np = (N + 127) // 128 * 128
    ldq = (9 * ((r + 8) // 9) + 127) // 128 * 128
    rb, cb, panels = Np // 128, ldq // 64, (Np // 128 + 1) // 2
    tiles = sum((rb - 2 * p) * cb for p in range(panels)) + sum(min(2 * p + 2, rb) * cb for p in range(panels))
    tiles += panels * (ldq // 128) * cb + ((ldq + 255) // 256) * rb * cb
    alg = 2.0 * N * N * r + 2.0 * N * r * r
    exe = tiles * 2.0 * 128 * 64 * 256 * 15
    pk, src = peaks()
    peak = pk["bf16_tflops_sustained"]
    roof = {"bound": "tensor", "achieved": alg / (ms_step / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": alg / (ms_step / 1e3) / 1e12 / peak, "traffic": None,
            "kernel": "ozaki_gemm (digit-split products with the inverse factor)",
            "peak_source": f"bf16 sustained ({src})",
            "work": f"2 N^2 r + 2 N r^2 = {alg:.3e} flop per update, N = {N}, r = 2k = {r}",
            "executed": {"flops_per_step": exe, "tflops": exe / (ms_step / 1e3) / 1e12,
                         "frac": exe / (ms_step / 1e3) / 1e12 / peak,
                         "what": "every 128x64 tile of the panel GEMMs x 15 digit products"},
            "timing": "work / whole update time (a lower bound of the GEMMs' rate)"}
    line = {"metric": "camera covariances/s after adding observations (4k-cam scene)", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == ccov.CCOV_PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "update", "cameras": scene.n, "points": scene.m, "observations": scene.t,
                       "added_observations": k, "precision": args.precision,
                       "step": "ccov_update_observations (device output) from the last step (d)",
                       "l2": "working set > L2: the inverse factor alone is "
                             f"{(9 * scene.n) ** 2 * 8 / 1e9:.1f} GB"},
            "clocks": clk,
            "e2e": {"value": scene.n * world / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": add.nbytes,
                    "d2h_bytes_per_step": scene.n * 81 * 8, "ms_per_step": ms_e2e},
            "gpu_launches": int(launches),
            "roofline": roof,
            "vs_new_step_d": {"ms_new_steps_a_to_d": ms_full, "speedup_of_update": ms_full / ms_step,
                              "max_rel_fro_per_block": float(errs["rel_fro"].max()),
                              "max_norm_err_per_block": float(errs["norm_err"].max()),
                              "max_pose_err_per_block": float(errs["pose_err"].max()),
                              "max_intr_err_per_block": float(errs["intr_err"].max())},
            "ms_by_added_observations": by_k}
    if rank == 0:
        print(json.dumps(line), flush=True)


UPDATE_K = 200
UPDATE_K_SWEEP = (20, 50, 800)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "subrecon":
        run_subrecon(args)
    elif args.workload == "surrogate":
        run_surrogate(args)
    elif args.workload == "update":
        run_update(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

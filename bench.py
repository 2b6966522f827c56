#!/usr/bin/env python3
"""Benchmark of the GPU FBP hot path (ramp filter + backprojection).

Workload (default): the float-vs-double configuration -- 512 x 512 image, 720
angles uniform on [0, pi), 725 detector bins, Shepp-Logan filter, sinograms of
20 seeded random ellipses with Poisson noise at I0 = 1e5 (log-transformed).  A
step reconstructs a batch of `--slices` such slices (distinct phantoms) that
are resident in HBM; their combined inputs, workspaces and images exceed the
129 MB L2.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

METRIC = "FBP slices/s and Gupdates/s (pixel×angle) vs plain path; serving p50/p99 ms"
FP32_LANES_PER_SM = 128
OPS_PER_UPDATE = 5  # FP32-pipe operations per pixel-angle update in the algorithmic count


def workload_spec(i: int) -> synthetic.SliceSpec:
    base = synthetic.cfg_float_double()
    return synthetic.SliceSpec(base.n_pix, base.n_angles, base.n_det, base.n_ellipses,
                               seed=base.seed + 1000 * i, filter=base.filter, i0=base.i0,
                               noise_seed=base.noise_seed + 1000 * i)


WORKLOAD_NAME = ("512x512 image, 720 angles on [0,pi), 725 bins, Shepp-Logan, "
                 "20 ellipses + Poisson I0=1e5 (float-vs-double configuration)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
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
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ reference arm
def cpu_fbp_time(specs, sinos, nthreads):
    import oracle
    theta = synthetic.default_angles(specs[0].n_angles)
    t0 = time.perf_counter()
    for spec, s in zip(specs, sinos):
        oracle.fbp(s, theta, spec.tau, spec.filter, spec.n_pix, nthreads=nthreads)
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    spec = workload_spec(0)
    sino = synthetic.sinogram(spec).astype(np.float32).astype(np.float64)
    for _ in range(args.warmup):
        cpu_fbp_time([spec], [sino], cores)
    times = []
    for _ in range(args.steps):
        times.append(cpu_fbp_time([spec], [sino], cores))
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "slices/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "gupdates_per_s": value * spec.updates / 1e9,
        "config": {"workload": WORKLOAD_NAME, "slices_per_step": 1,
                   "l2": "host run (no GPU)"},
        "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores, "kind": "oracle",
                         "sample": "one full 512x512x720 slice per step (FP64 C oracle, "
                                   "filter + backprojection, all host cores)"},
        "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2109_02174_gb300 as fbp
    from paper_2109_02174_gb300 import build as fbp_build

    if rank == 0 or not os.path.exists(fbp.LIB_PATH):
        fbp_build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    S = args.slices
    specs = [workload_spec(rank * S + i) for i in range(S)]
    spec0 = specs[0]
    theta = synthetic.default_angles(spec0.n_angles)
    host = [synthetic.sinogram(s, theta).astype(np.float32) for s in specs]
    plan = fbp.Plan(spec0.n_pix, spec0.n_angles, spec0.n_det, filter=spec0.filter)
    sinos = [torch.from_numpy(h).to(dev) for h in host]
    works = [plan.empty_workspace() for _ in range(S)]
    images = [plan.empty_image() for _ in range(S)]
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    ld = spec0.n_det
    resident_mb = S * (spec0.n_angles * spec0.n_det * 4 + plan.workspace_bytes +
                       spec0.n_pix ** 2 * 4) / 1e6

    def step(ev=None):
        for i in range(S):
            fbp.fbp_filter(plan.handle, sinos[i].data_ptr(), ld, works[i].data_ptr(), sp)
            if ev is not None:
                ev[i][0].record(stream)
            fbp.fbp_backproject(plan.handle, works[i].data_ptr(), images[i].data_ptr(), sp)
            if ev is not None:
                ev[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.device_status()

    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
           for _ in range(S)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = t_start.elapsed_time(t_end)
    bp_ms = [ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps) for i in range(S)]
    plan.device_status()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the C ABI with host buffers: pinned sinograms in, images out
    h_sino = [torch.from_numpy(h).pin_memory() for h in host]
    h_img = [torch.empty((spec0.n_pix, spec0.n_pix), dtype=torch.float32).pin_memory()
             for _ in range(S)]

    def e2e_step():
        for i in range(S):
            sinos[i].copy_(h_sino[i], non_blocking=True)
            fbp.fbp_reconstruct(plan.handle, sinos[i].data_ptr(), ld, images[i].data_ptr(),
                                works[i].data_ptr(), sp)
            h_img[i].copy_(images[i], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())

    if rank != 0:
        return 0
    total_slices = S * args.steps * world
    value = total_slices / (ms / 1e3)
    upd = spec0.updates
    pk, pk_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_gups = FP32_LANES_PER_SM * sms * sm_mhz * 1e6 / OPS_PER_UPDATE / 1e9
    bp_mean = sum(bp_ms) / len(bp_ms)
    achieved = upd / (bp_mean / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "gupdates_per_s": value * upd / 1e9,
        "config": {"workload": WORKLOAD_NAME, "slices_per_step": S * world,
                   "path": "plain single-slice calls (fbp_filter + fbp_backproject per slice)",
                   "l2": f"inputs larger than L2: {resident_mb:.0f} MB resident per GPU",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "bp_f32_kernel", "achieved": achieved,
                     "peak": peak_gups, "unit": "Gupdates/s", "frac": achieved / peak_gups,
                     "traffic": None,
                     "peak_basis": f"{FP32_LANES_PER_SM} FP32 lanes x {sms} SMs x {sm_mhz:.0f} "
                                   f"MHz ({pk_kind} sm_max_mhz) / {OPS_PER_UPDATE} FP32 ops per "
                                   f"update",
                     "launch_ms": bp_mean},
        "e2e": {"value": total_slices / (e2e_ms / 1e3), "unit": "slices/s",
                "h2d_bytes_per_step": S * spec0.n_angles * spec0.n_det * 4,
                "d2h_bytes_per_step": S * spec0.n_pix ** 2 * 4},
        "gpu_launches": 2 * S * args.steps,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = [host[0].astype(np.float64)]
        t = cpu_fbp_time([spec0], sample, cores)
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": "slices/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "one full slice of the workload (FP64 C oracle, "
                                          "filter + backprojection, all host cores)"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--slices", type=int, default=64)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

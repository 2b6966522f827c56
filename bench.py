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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

METRIC = "FBP slices/s and Gupdates/s (pixel×angle) vs plain path; serving p50/p99 ms"
FP32_LANES_PER_SM = 128
OPS_PER_UPDATE = 5  # FP32-pipe operations per pixel-angle update in the algorithmic count
FILTER_PATHS = {"auto": 0, "tc": 1, "fft": 2, "direct": 3}
# Shared-memory ceiling of the backprojection: every update loads one 8-byte
# (mid, slope) pair, and a warp's 8-byte shared load moves two 128-byte
# wavefronts, so at most 16 updates per clock per SM.
SMEM_UPDATES_PER_CLK_SM = 16
# DRAM bytes (read + write) of one backprojection launch, measured by ncu on
# the launch this script times for the shape the tuner picks
# (profiles/bp_persistent_kernel_batch64_512x720x725.md),
# keyed by (geometry, slices, tile_x, tile_y, angle_chunk); reported only when
# the tuned launch is that one, null otherwise.
BP_TRAFFIC = {("512x720x725", 64, 32, 32, 32): 247432960 + 55667968}
ROUTE_NAMES = {1: "tensor-core Toeplitz", 2: "FFT", 3: "direct-convolution"}


def workload_spec(i: int) -> synthetic.SliceSpec:
    return synthetic.cfg_float_double_slice(i)


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
    """SM clock and clock-event reasons of one GPU, sampled every 5 ms from a
    thread through NVML (read-only queries) while the timed region runs;
    nvidia-smi every 10 ms if NVML cannot be loaded."""
    PERIOD_S = 0.005
    # nvmlClocksEventReason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, props=None):
        self.gpu = gpu_index
        self.props = props
        self.samples = []
        self.proc = None
        self.thread = None
        self.nvml = None
        self.handle = None
        self.max_mhz = None
        self.path = os.path.join(tempfile.gettempdir(), f"fbp_clocks_{os.getpid()}.csv")

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            ok = False
            p = self.props
            if p is not None and hasattr(p, "pci_bus_id"):
                bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) == 0
            if not ok:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) == 0
            if not ok:
                return False
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.nvml, self.handle = lib, h
            return True
        except Exception:
            return False

    def _loop(self):
        import ctypes
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self.stop_flag:
            if self.nvml.nvmlDeviceGetClockInfo(self.handle, 1, ctypes.byref(clk)) == 0:
                r = rs.value if self.reason_fn(self.handle, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), int(r)))
            time.sleep(self.PERIOD_S)

    def start(self):
        import threading
        self.samples = []
        self.stop_flag = False
        if self.nvml is not None or self._nvml_open():
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "10"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag = True
            self.thread.join(timeout=5)
            self.thread = None
            if not self.samples:
                return None
            sm = [c for c, _ in self.samples]
            reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items()
                              if r & bit})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "nvml, 5 ms"}
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
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi, 10 ms"}


# ------------------------------------------------------------------ reference arm
def cpu_fbp_time(specs, sinos, nthreads):
    import oracle
    theta = synthetic.default_angles(specs[0].n_angles)
    t0 = time.perf_counter()
    for spec, s in zip(specs, sinos):
        oracle.fbp(s, theta, spec.tau, spec.filter, spec.n_pix, nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_config_times(cores):
    """The FP64 oracle once on the batched configuration's 64 uneven slices and
    once on the large slice (2048^2, 2048 angles, 2899 bins), all host cores:
    slices/s and Gupdates/s beside the GPU's."""
    import oracle
    out = {}
    for name, specs in (("batched_uneven_64", synthetic.cfg_batch()),
                        ("large_2048x2048x2899", [synthetic.cfg_large()])):
        thetas = [synthetic.default_angles(s.n_angles) for s in specs]
        sinos = [synthetic.sinogram(s, th).astype(np.float32).astype(np.float64)
                 for s, th in zip(specs, thetas)]
        t0 = time.perf_counter()
        for s, th, sino in zip(specs, thetas, sinos):
            oracle.fbp(sino, th, s.tau, s.filter, s.n_pix, nthreads=cores)
        sec = time.perf_counter() - t0
        out[name] = {"slices_per_s": len(specs) / sec,
                     "gupdates_per_s": sum(s.updates for s in specs) / sec / 1e9,
                     "seconds": sec}
    return out


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


# ------------------------------------------------------------------ ranks
def shard_ids(rank: int, world: int, per_rank: int) -> list[int]:
    """Slice ids of one rank: replicas with disjoint phantoms (weak scaling,
    no data exchanged between ranks)."""
    return [rank * per_rank + i for i in range(per_rank)]


def max_over_ranks(value: float, world: int, device) -> float:
    """The timed region's length over all ranks (the slowest rank)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ our arm
def _timed(fn, steps, stream, per_launch=False):
    """Run fn() `steps` times between CUDA events on `stream`; returns total ms
    (and the per-launch ms list when per_launch)."""
    import torch
    if per_launch:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        per = [a.elapsed_time(b) for a, b in evs]
        return sum(per), per
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


SERVE_CHECK_EVERY = 100  # one request in 100 (1%) is checked against alone and the oracle


def pinned_views(shapes):
    """Float32 host tensors of the given shapes, all views of ONE pinned
    allocation (256-byte aligned each).  Thousands of separate pinned
    allocations made the server's per-request copies measurably slower (p99
    0.83 -> 1.12 ms over four serving runs in one process)."""
    import torch
    sizes = [int(np.prod(sh)) for sh in shapes]
    offs, total = [], 0
    for n in sizes:
        offs.append(total)
        total += (n + 63) // 64 * 64
    slab = torch.empty(max(total, 1), dtype=torch.float32).pin_memory()
    return [slab[o:o + n].view(*sh) for o, n, sh in zip(offs, sizes, shapes)]


def prepare_serving(seconds: float, rate: float = 2000.0):
    """Inputs of the serving run, made before any timed region (tens of
    seconds of CPU work on every core just before the serving loop raised its
    p99): the arrival stream, the pool of two seeded noisy phantoms per
    geometry, and the sampled requests' own seeded sinograms, all pinned."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    count = int(seconds * rate)
    stream = synthetic.serving_stream(count, seed=5, rate=rate)
    geoms = sorted({(s.n_pix, s.n_angles, s.n_det) for _, s in stream})
    pool_np = {}
    for g in geoms:
        pool_np[g] = []
        for k in range(2):
            spec = synthetic.SliceSpec(g[0], g[1], g[2], 10, seed=50000 + 97 * k + g[0] + g[1],
                                       i0=1e5, noise_seed=150000 + 97 * k + g[0] + g[1])
            pool_np[g].append(synthetic.sinogram(spec).astype(np.float32))
    sampled = [k for k in range(count) if k % SERVE_CHECK_EVERY == 0]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        own = dict(zip(sampled, ex.map(
            lambda k: synthetic.sinogram(stream[k][1]).astype(np.float32), sampled)))
    RING = 48
    sizes = sorted({g[0] for g in geoms})
    shapes = ([a.shape for g in geoms for a in pool_np[g]] + [own[k].shape for k in sampled] +
              [(stream[k][1].n_pix,) * 2 for k in sampled] + [(n, n) for n in sizes
                                                              for _ in range(RING)])
    views = iter(pinned_views(shapes))
    pool = {}
    for g in geoms:
        pool[g] = []
        for a in pool_np[g]:
            v = next(views)
            v.copy_(torch.from_numpy(a))
            pool[g].append(v)
    own_pinned = {}
    for k in sampled:
        v = next(views)
        v.copy_(torch.from_numpy(own[k]))
        own_pinned[k] = v
    own_out = {k: next(views) for k in sampled}
    rings = {n: [next(views) for _ in range(RING)] for n in sizes}
    return {"rate": rate, "count": count, "stream": stream, "geoms": geoms, "pool": pool,
            "own": own, "own_pinned": own_pinned, "own_out": own_out, "rings": rings,
            "ring": RING}


def run_serving(fbp, prep, budget_gb: float = 40.0, max_wave: int = 32, n_streams: int = 3):
    """Poisson arrivals (mean 2000/s, exponential gaps from SplitMix64(5)) of
    slices with n in {256,512,768,1024}, A in {360,720,1440}, D = ceil(n sqrt2)+1,
    noisy (I0 = 1e5), inputs from prepare_serving.  One request in 100 carries
    its own seeded sinogram (phantom seed 50000 + r, noise seed 150000 + r) and
    its own output buffer; it is compared bit for bit with its alone result and
    kept for the oracle check (check_serving_sample, run last).  The other
    requests' sinograms come from a pool of two seeded phantoms per geometry
    (generating 2 x 10^4 distinct analytic sinograms would take longer than the
    run); every request has its own pinned output slot.  After the arrival run,
    the capacity: the first 4000 requests submitted as fast as output slots free
    up, through the server and, for the plain single-slice path, one
    fbp_reconstruct per request with its host-to-device and device-to-host
    copies on one stream."""
    import torch
    rate, stream, geoms, pool = prep["rate"], prep["stream"], prep["geoms"], prep["pool"]
    own, own_pinned, own_out = prep["own"], prep["own_pinned"], prep["own_out"]
    RING, rings = prep["ring"], prep["rings"]
    owner = {n: [None] * RING for n in rings}
    # warm-up: one request per geometry through a throw-away server, so kernel
    # loading and first-touch costs stay out of the measured run
    warm = fbp.Server(1 << 30, max_wave=max_wave, n_streams=n_streams)
    for g in geoms:
        wid = warm.submit(pool[g][0], rings[g[0]][0], g[0])
        warm.wait(wid, 60.0)
    warm.close()
    server = fbp.Server(int(budget_gb * (1 << 30)), max_wave=max_wave, n_streams=n_streams)
    for g in geoms:
        server.warm(g[0], g[1], g[2])
    counters = {n: 0 for n in rings}
    check = {}
    # the load generator is this Python loop: a cyclic garbage collection of
    # the run's tens of thousands of objects would pause it for tens of ms
    # and show up as server latency (one run: p99 21 ms, max 36 ms)
    import gc
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    for k, (t, spec) in enumerate(stream):
        n = spec.n_pix
        slot = counters[n] % RING
        counters[n] += 1
        if owner[n][slot] is not None:
            server.wait(owner[n][slot], 60.0)
        while True:
            dt = t - (time.perf_counter() - t0)
            if dt <= 0:
                break
            if dt > 2e-4:
                time.sleep(dt - 1e-4)
        if k in own_pinned:  # sampled request: own sinogram and output buffer
            rid = server.submit(own_pinned[k], own_out[k], n)
            check[k] = own_out[k]
        else:
            g = (n, spec.n_angles, spec.n_det)
            rid = server.submit(pool[g][k % 2], rings[n][slot], n)
            owner[n][slot] = rid
    server.drain(300.0)
    gc.enable()
    st = server.stats()
    # the sampled requests against their alone results, bit for bit
    plans = {}
    equal = 0
    for k, out in check.items():
        spec = stream[k][1]
        g = (spec.n_pix, spec.n_angles, spec.n_det)
        if g not in plans:
            plans[g] = fbp.Plan(*g, tile_x=-1, tile_y=-1)  # the server's plan choice
        alone = plans[g].reconstruct(own_pinned[k].cuda())
        torch.cuda.synchronize()
        equal += int(torch.equal(alone.cpu(), out))
    server.close()
    # capacity: the same request mix submitted as fast as output slots free up
    # (up to 48 per image size in flight), timed from the first submit to the
    # last completion
    burst = stream[:4000]

    def saturate(budget_bytes):
        sat = fbp.Server(int(budget_bytes), max_wave=max_wave, n_streams=n_streams)
        for g in geoms:
            sat.warm(g[0], g[1], g[2])
        owner = {n: [None] * RING for n in rings}
        counters = {n: 0 for n in rings}
        t_sat = time.perf_counter()
        for k, (_, spec) in enumerate(burst):
            n = spec.n_pix
            slot = counters[n] % RING
            counters[n] += 1
            if owner[n][slot] is not None:
                sat.wait(owner[n][slot], 60.0)
            owner[n][slot] = sat.submit(pool[(n, spec.n_angles, spec.n_det)][k % 2],
                                        rings[n][slot], n)
        sat.drain(300.0)
        t_sat = time.perf_counter() - t_sat
        sst = sat.stats()
        sat.close()
        return t_sat, sst
    t_sat, sst = saturate(budget_gb * (1 << 30))
    # the same burst under a budget that binds (a few of the largest requests,
    # 29 MB each, at a time): admission stalls, and what they cost
    tight_gb = 0.25
    t_tight, tst = saturate(tight_gb * (1 << 30))
    # the plain single-slice path on the same 4000 requests: per request the
    # sinogram copy in, one fbp_reconstruct (default plan of its geometry), the
    # image copy out, all on one stream
    cs = torch.cuda.current_stream()
    sp = int(cs.cuda_stream)
    pplans = {g: fbp.Plan(*g) for g in geoms}
    dsino = {g: torch.empty((g[1], g[2]), device="cuda") for g in geoms}
    dimg = {g: torch.empty((g[0], g[0]), device="cuda") for g in geoms}
    dws = {g: pplans[g].empty_workspace() for g in geoms}

    def plain_request(k, spec):
        g = (spec.n_pix, spec.n_angles, spec.n_det)
        dsino[g].copy_(pool[g][k % 2], non_blocking=True)
        fbp.fbp_reconstruct(pplans[g].handle, dsino[g].data_ptr(), g[2], dimg[g].data_ptr(),
                            dws[g].data_ptr(), sp)
        rings[g[0]][k % RING].copy_(dimg[g], non_blocking=True)
    for g in geoms:  # first call per geometry outside the timing
        plain_request(0, synthetic.SliceSpec(g[0], g[1], g[2], 1, 0))
    torch.cuda.synchronize()
    t_plain = time.perf_counter()
    for k, (_, spec) in enumerate(burst):
        plain_request(k, spec)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t_plain
    upd = sum(s.updates for _, s in stream)
    sat_upd = sum(s.updates for _, s in burst)
    capacity = {"requests": sst["completed"], "seconds": t_sat,
                "slices_per_s": sst["completed"] / t_sat,
                "gupdates_per_s": sat_upd / t_sat / 1e9,
                "p50_ms": sst["p50_ms"], "p99_ms": sst["p99_ms"],
                "max_waves_in_flight": sst["max_waves_in_flight"],
                "plain_path_slices_per_s": len(burst) / t_plain,
                "plain_path": "one fbp_reconstruct per request (default plan), sinogram "
                              "copied in and image copied out, one stream, same 4000 requests",
                "what": "the first 4000 requests of the mix, submitted without arrival gaps",
                "tight_budget": {"budget_gb": tight_gb, "slices_per_s": tst["completed"] / t_tight,
                                 "admission_stalls": tst["admission_stalls"],
                                 "peak_gb": tst["peak_bytes"] / 2 ** 30,
                                 "p50_ms": tst["p50_ms"], "p99_ms": tst["p99_ms"],
                                 "what": "the same 4000 requests with a 0.25 GB arena"}}
    result = {
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
        "max_ms": st["max_ms"], "requests": st["completed"], "failed": st["failed"],
        "slices_per_s": st["completed"] / st["span_s"] if st["span_s"] else None,
        "gupdates_per_s": upd / st["span_s"] / 1e9 if st["span_s"] else None,
        "offered_rate_per_s": rate, "offered_seconds": stream[-1][0],
        "admission_stalls": st["admission_stalls"], "waves": st["waves"],
        "max_waves_in_flight": st["max_waves_in_flight"],
        "peak_gb": st["peak_bytes"] / 2 ** 30, "budget_gb": budget_gb,
        "bitwise_equal_to_alone": f"{equal}/{len(check)} sampled requests "
                                  f"(1 in {SERVE_CHECK_EVERY}, own seeded sinograms)",
        "latency": "submit to the end of the image copy to pinned host memory",
        "capacity": capacity,
    }
    sample = [(stream[k][1], own[k], check[k].numpy().copy()) for k in sorted(check)]
    return result, sample


def check_serving_sample(sample, cores):
    """The sampled serving results against the FP64 oracle's whole images
    (all host cores): how many meet the FP32 bars, and the worst errors."""
    import oracle
    ok, worst_max, worst_rmse = 0, 0.0, 0.0
    t0 = time.perf_counter()
    for spec, sino32, img in sample:
        th = synthetic.default_angles(spec.n_angles)
        ref = oracle.fbp(sino32.astype(np.float64), th, spec.tau, spec.filter, spec.n_pix,
                         nthreads=cores)
        scale = float(np.abs(ref).max())
        err = img.astype(np.float64) - ref
        e_max = float(np.abs(err).max()) / scale
        e_rms = float(np.sqrt(np.mean(err ** 2))) / scale
        ok += int(e_max <= 1e-4 and e_rms <= 2e-5)
        worst_max, worst_rmse = max(worst_max, e_max), max(worst_rmse, e_rms)
    return {"within_fp32_bars": f"{ok}/{len(sample)}", "worst_max_rel": worst_max,
            "worst_rmse_rel": worst_rmse, "seconds": time.perf_counter() - t0,
            "what": "every pixel of each sampled request against the FP64 oracle's image"}


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 rate (nominal; no measured figure on this machine)
# FP64 instructions per update of the FP64 backprojection: the interpolating FMA
# and the sum (the detector coordinate is integer fixed point)
FP64_OPS_PER_UPDATE = 2
# SSIM on the device: per window 2 x 5 x 11 FP64 FMAs (the separable 11-tap
# Gaussian, rows then columns, over x, y, x^2 + y^2, d, d^2) and about 10 for
# the window's formula
QUALITY_FP64_PER_WINDOW = 120


def _timed_flushed(fn, steps, stream, flush):
    """Time fn() `steps` times with CUDA events around each call only, writing
    `flush` (larger than L2) before each, so every call starts with a cold L2.
    Returns the mean ms per call."""
    import torch
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def run_configs(fbp):
    """Per-configuration figures beside the headline, one slice per call
    through fbp_reconstruct (the plain path), L2 flushed before each call:
    the plain slice (256^2, 180 angles, 363 bins, Ram-Lak, FFT length 1024),
    the float-vs-double slice on the FP64 path (against the nominal FP64 rate),
    PSNR/SSIM (on the GPU) of the FP32, Kahan and FP16-pair images of the
    float-vs-double slice against its FP64 image; and the large slice
    (2048^2, 2048 angles, 2899 bins) with the filter time
    of the FFT and tensor-core routes and the speed of its FP16-pair and Kahan
    variants; the batched filter of 64 float-vs-double slices fed line
    integrals or photon counts (Lambert-Beer conversion on load); and a volume
    interpolated from a stack of 64 slices."""
    import torch
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}

    def one_slice(spec, dtype=0, reps=20, **opt):
        plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter, dtype=dtype,
                        **opt)
        host = synthetic.sinogram(spec)
        sino = torch.from_numpy(host if dtype == 1 else host.astype(np.float32)).cuda()
        img, ws = plan.empty_image(), plan.empty_workspace()

        def call():
            fbp.fbp_reconstruct(plan.handle, sino.data_ptr(), sino.stride(0), img.data_ptr(),
                                ws.data_ptr(), sp)
        call()
        torch.cuda.synchronize()
        plan.device_status()
        ms = _timed_flushed(call, reps, stream, flush)
        return plan, sino, ms

    spec = synthetic.cfg_plain()
    _, _, ms = one_slice(spec, fft_len=1024)
    out["plain_256x180x363"] = {"ms_per_slice": ms, "slices_per_s": 1e3 / ms,
                                "gupdates_per_s": spec.updates / (ms / 1e3) / 1e9,
                                "path": "fbp_reconstruct, FP32, FFT length 1024"}
    spec = synthetic.cfg_float_double()
    p64, s64, ms = one_slice(spec, dtype=1, reps=5)
    gups = spec.updates / (ms / 1e3) / 1e9
    # the paper's comparison measures (Eqs. 3, 4) on the device: each FP32
    # variant's image against the FP64 path's image of the same slice
    img64 = p64.reconstruct(s64).float()
    s32 = s64.float()
    quality = {}
    for name, opt in (("fp32", {}), ("fp32_kahan", {"accumulate": 1}),
                      ("fp16_pairs", {"q_storage": 2})):
        img = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                       **opt).reconstruct(s32)
        db, ss = fbp.quality(img, img64)
        quality[name] = {"psnr_db": db, "ssim": ss, "one_minus_ssim": 1.0 - ss}
    # the quality call itself (PSNR and SSIM of one 512^2 pair), L2 flushed:
    # FP64 work, about QUALITY_FP64_PER_WINDOW instructions per SSIM window
    # (the 11-tap separable Gaussian over five maps, twice, and the formula)
    import ctypes
    qn = spec.n_pix
    qbytes = ctypes.c_size_t()
    lib = fbp.load_library()
    lib.fbp_quality_scratch_bytes(qn, qn, ctypes.byref(qbytes))
    qscr = torch.empty(max(int(qbytes.value), 16), dtype=torch.uint8, device="cuda")
    qout = torch.empty(2, dtype=torch.float64, device="cuda")
    sp_q = int(torch.cuda.current_stream().cuda_stream)

    def quality_call():
        lib.fbp_quality(img.data_ptr(), img64.data_ptr(), qn, qn, qn, ctypes.c_double(0.0),
                        qscr.data_ptr(), ctypes.c_size_t(qscr.numel()), qout.data_ptr(), sp_q)
    quality_call()
    torch.cuda.synchronize()
    qms = _timed_flushed(quality_call, 10, torch.cuda.current_stream(), flush)
    windows = (qn - 10) ** 2
    q_peak = FP64_NOMINAL_TFLOPS * 1e12 / 2 / QUALITY_FP64_PER_WINDOW  # windows/s
    quality["timing"] = {"us": qms * 1e3, "windows": windows,
                         "windows_per_s": windows / (qms / 1e3),
                         "frac_of_fp64_peak": windows / (qms / 1e3) / q_peak,
                         "peak_basis": "nominal 1.25 TFLOP/s FP64 = 0.625 T FP64 "
                                       "instructions/s, %d per window" %
                                       QUALITY_FP64_PER_WINDOW}
    out["quality_vs_fp64_512x720x725"] = quality
    fp64_peak = FP64_NOMINAL_TFLOPS * 1e12 / 2 / FP64_OPS_PER_UPDATE / 1e9
    out["fp64_512x720x725"] = {"ms_per_slice": ms, "slices_per_s": 1e3 / ms,
                               "gupdates_per_s": gups, "fp64_peak_gupdates_per_s": fp64_peak,
                               "frac_of_fp64_peak": gups / fp64_peak,
                               "filter": ROUTE_NAMES.get(p64.filter_path, "?") + " (FP64)",
                               "peak_basis": "nominal 1.25 TFLOP/s FP64 = 0.625 T FP64 "
                                             "instructions/s, 2 per update (lerp FMA, sum); "
                                             "the time includes the FP64 filter"}
    spec = synthetic.cfg_large()
    plan, sino, ms = one_slice(spec, reps=5)
    entry = {"ms_per_slice": ms, "slices_per_s": 1e3 / ms,
             "gupdates_per_s": spec.updates / (ms / 1e3) / 1e9, "filter_ms": {}}
    for name, path in (("fft", 2), ("tc", 1)):
        fp = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                      filter_path=path)
        q = fp.empty_filtered()

        def filt():
            fbp.fbp_filter(fp.handle, sino.data_ptr(), sino.stride(0), q.data_ptr(), sp)
        filt()
        torch.cuda.synchronize()
        entry["filter_ms"][name] = _timed_flushed(filt, 5, stream, flush)
    # the backprojection launch of the large slice alone (one slice, the
    # default plan's tile), against the ALU figure and the shared-memory
    # ceiling of the headline's roofline record
    q_large = plan.filter(sino)
    img_large = plan.empty_image()

    def bp_large():
        fbp.fbp_backproject(plan.handle, q_large.data_ptr(), img_large.data_ptr(), sp)
    bp_large()
    torch.cuda.synchronize()
    bp_ms = _timed_flushed(bp_large, 10, stream, flush)
    pk_l, pk_kind_l = peaks()
    sms_l = torch.cuda.get_device_properties(0).multi_processor_count
    mhz_l = float(pk_l.get("sm_max_mhz", 2070.0))
    peak_l = FP32_LANES_PER_SM * sms_l * mhz_l * 1e6 / OPS_PER_UPDATE / 1e9
    smem_l = SMEM_UPDATES_PER_CLK_SM * sms_l * mhz_l / 1e3
    ach_l = spec.updates / (bp_ms / 1e3) / 1e9
    entry["roofline"] = {
        "bound": "alu", "kernel": "bp_persistent_kernel (one slice, default plan)",
        "achieved": ach_l, "peak": peak_l, "unit": "Gupdates/s", "frac": ach_l / peak_l,
        "smem_ceiling": {"gupdates_per_s": smem_l, "frac": ach_l / smem_l},
        "launch_ms": bp_ms, "updates_per_launch": spec.updates,
        "traffic": None, "peak_basis": f"as the headline ({pk_kind_l} sm_max_mhz)"}
    del q_large, img_large
    # the Lambert-Beer conversion fused into the filter's loads: the batched
    # filter of 64 float-vs-double slices from line integrals and from counts
    fb = synthetic.cfg_float_double()
    lb = {}
    for name, i0 in (("line_integrals", 0.0), ("photon_counts", fb.i0)):
        fp = fbp.Plan(fb.n_pix, fb.n_angles, fb.n_det, filter=fb.filter, filter_path=2, i0=i0)
        src = [torch.full((fb.n_angles, fb.n_det), 5000.0, device="cuda") for _ in range(64)]
        fbatch = fbp.Batch([fp] * 64, src, parts=fbp.FBP_BATCH_FILTER)
        fbatch.launch()
        torch.cuda.synchronize()
        lb[name] = _timed_flushed(fbatch.launch, 5, stream, flush) / 64 * 1e3
        fbatch.close()
    out["lambert_beer_on_load_us_per_slice"] = lb
    # FDK cone-beam (the paper's future work): 256^3 voxels, 360 angles over a
    # full turn, 448 x 320 detector, source radius 1024 voxels
    fdk_plan = fbp.FdkPlan(360, 320, 448, 1024.0, 256, 256, 256)
    proj = torch.randn((360, 320, 448), device="cuda")
    fvol = torch.empty((256, 256, 256), device="cuda")
    fws = torch.empty(fdk_plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    fdk_plan.reconstruct(proj, fvol, fws)
    torch.cuda.synchronize()
    fms = _timed_flushed(lambda: fdk_plan.reconstruct(proj, fvol, fws), 3, stream, flush)
    fupd = 256 ** 3 * 360
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(peaks()[0].get("sm_max_mhz", 2070.0))
    smem_ceiling = 8 * sms * mhz / 1e3  # two 8-byte shared loads per update: 8 updates/clk/SM
    out["fdk_256cubed_360x320x448"] = {
        "ms": fms, "voxel_updates_per_s": fupd / (fms / 1e3),
        "gupdates_per_s": fupd / (fms / 1e3) / 1e9,
        "smem_ceiling_gupdates_per_s": smem_ceiling,
        "frac_of_smem_ceiling": fupd / (fms / 1e3) / 1e9 / smem_ceiling,
        "what": "weight + FFT filter of 115200 rows + TMA-staged backprojection"}
    fdk_plan.close()
    # a volume from a stack of 64 reconstructed 512^2 slices, four planes per
    # gap (253 planes): an HBM-bound stream; minimal bytes = slices read once
    # + planes written once
    import ctypes
    K, n = 64, 512
    zs = np.arange(K, dtype=np.float64)
    zo = np.linspace(0.0, K - 1.0, 4 * (K - 1) + 1)
    slices = [torch.randn((n, n), device="cuda") for _ in range(K)]
    vol = torch.empty((zo.size, n, n), device="cuda")
    c_ptrs = (ctypes.c_void_p * K)(*[t.data_ptr() for t in slices])
    c_z = (ctypes.c_double * K)(*zs)
    c_zo = (ctypes.c_double * zo.size)(*zo)
    lib = fbp.load_library()

    def vol_call():
        lib.fbp_volume_from_slices(c_ptrs, K, c_z, n, c_zo, zo.size, vol.data_ptr(), sp)
    vol_call()
    torch.cuda.synchronize()
    vms = _timed_flushed(vol_call, 5, stream, flush)
    vbytes = (K + zo.size) * n * n * 4
    pk, _ = peaks()
    out["volume_64x512_to_253_planes"] = {
        "ms": vms, "gb_per_s_min_bytes": vbytes / (vms / 1e3) / 1e9,
        "hbm_peak_gbs": pk["hbm_gbs"],
        "frac_of_hbm": vbytes / (vms / 1e3) / 1e9 / pk["hbm_gbs"],
        "min_bytes": vbytes}
    entry["variants_gupdates_per_s"] = {}
    for name, opt in (("fp16_pairs", {"q_storage": 2}), ("kahan", {"accumulate": 1})):
        _, _, vms = one_slice(spec, reps=5, **opt)
        entry["variants_gupdates_per_s"][name] = spec.updates / (vms / 1e3) / 1e9
    out["large_2048x2048x2899"] = entry
    return out


def run_uneven(fbp, plan_cache=None):
    """The batched configuration: 64 uneven slices (n from {256,384,512,768},
    A from {180,360,720,1440}, D = ceil(n sqrt2)+1, seeds 1000+s) in one graph,
    against the same slices through one fbp_reconstruct call each."""
    import torch
    specs = synthetic.cfg_batch()
    plans = {}
    for s in specs:
        key = (s.n_pix, s.n_angles, s.n_det)
        if key not in plans:
            # each shape tuned (filter route, tile, angle chunk) for a batch of 64
            plans[key] = fbp.Plan(*key, filter=s.filter, autotune=True, batch_hint=len(specs))
    pl = [plans[(s.n_pix, s.n_angles, s.n_det)] for s in specs]
    sinos = [torch.from_numpy(synthetic.sinogram(s).astype(np.float32)).cuda() for s in specs]
    batch = fbp.Batch(pl, sinos)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        batch.launch()
    torch.cuda.synchronize()
    steps = 10
    ms = _timed(batch.launch, steps, stream)
    batch.status()

    def one_by_one():
        for p, s, img, ws in zip(pl, sinos, batch.images, batch.workspaces):
            fbp.fbp_reconstruct(p.handle, s.data_ptr(), s.stride(0), img.data_ptr(),
                                ws.data_ptr(), int(stream.cuda_stream))
    one_by_one()
    plain_ms = _timed(one_by_one, steps, stream)
    upd = sum(s.updates for s in specs)
    batch.close()
    return {"slices": len(specs), "slices_per_s": len(specs) * steps / (ms / 1e3),
            "gupdates_per_s": upd * steps / (ms / 1e3) / 1e9,
            "plain_path_slices_per_s": len(specs) * steps / (plain_ms / 1e3),
            "what": "cfg recipe: 64 slices, n in {256,384,512,768}, A in {180,360,720,1440}, "
                    "plans autotuned per shape for a batch of 64, one captured graph per step"}


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
    serve_prep = None
    if world == 1 and args.serve_seconds > 0:
        serve_prep = prepare_serving(args.serve_seconds)
    S = args.slices
    specs = [workload_spec(i) for i in shard_ids(rank, world, S)]
    spec0 = specs[0]
    theta = synthetic.default_angles(spec0.n_angles)
    host = [synthetic.sinogram(s, theta).astype(np.float32) for s in specs]
    # the autotuner picks the filter route and backprojection shape for this
    # geometry on this GPU (timed over a batch; cached in FBP_TUNE_CACHE if set)
    shape = {}
    if args.tile:
        tx, ty = (int(v) for v in args.tile.split("x"))
        shape = {"tile_x": tx, "tile_y": ty, "angle_chunk": args.chunk}
    plan = fbp.Plan(spec0.n_pix, spec0.n_angles, spec0.n_det, filter=spec0.filter,
                    autotune=True, batch_hint=min(S, 64),
                    filter_path=FILTER_PATHS[args.filter_path], **shape)
    sinos = [torch.from_numpy(h).to(dev) for h in host]
    works = [plan.empty_workspace() for _ in range(S)]
    images = [plan.empty_image() for _ in range(S)]
    plans = [plan] * S
    full = fbp.Batch(plans, sinos, images, works)
    bp_only = fbp.Batch(plans, sinos, images, works, parts=fbp.FBP_BATCH_BACKPROJECT)
    filt_only = fbp.Batch(plans, sinos, images, works, parts=fbp.FBP_BATCH_FILTER)
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    ld = spec0.n_det
    resident_mb = S * (spec0.n_angles * spec0.n_det * 4 + plan.workspace_bytes +
                       spec0.n_pix ** 2 * 4) / 1e6

    for _ in range(args.warmup):
        full.launch()
    torch.cuda.synchronize()
    full.status()

    # ---- timed region: K steps of the batched hot path (filter + backprojection)
    clocks = ClockSampler(local_rank, torch.cuda.get_device_properties(dev))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ms = _timed(full.launch, args.steps, stream)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(ms, world, dev)
    full.status()

    # ---- the backprojection launch alone over the same buffers (roofline)
    bp_only.launch()
    _, bp_ms = _timed(bp_only.launch, max(args.steps // 4, 5), stream, per_launch=True)
    filt_only.launch()
    filt_ms = _timed(filt_only.launch, max(args.steps // 4, 5), stream) / max(args.steps // 4, 5)

    # ---- serving, early: later in the same process its p99 rose (0.83 ms in a
    # fresh process, 1.0-1.5 ms after the other measurements)
    serve_result = serve_sample = None
    if serve_prep is not None:
        serve_result, serve_sample = run_serving(fbp, serve_prep)

    # ---- the plain single-slice path (one fbp_reconstruct call per slice)
    def plain_step():
        for i in range(S):
            fbp.fbp_reconstruct(plan.handle, sinos[i].data_ptr(), ld, images[i].data_ptr(),
                                works[i].data_ptr(), sp)
    plain_step()
    plain_steps = max(args.steps // 10, 3)
    plain_ms = _timed(plain_step, plain_steps, stream)

    # ---- end to end through the C ABI from pinned host buffers
    pv = pinned_views([h.shape for h in host] + [(spec0.n_pix, spec0.n_pix)] * S)
    h_sino, h_img = pv[:S], pv[S:]
    for hs, h in zip(h_sino, host):
        hs.copy_(torch.from_numpy(h))
    full.run_host(h_sino, h_img)
    torch.cuda.synchronize()
    e2e_steps = max(args.steps // 4, 5)
    e2e_ms = _timed(lambda: full.run_host(h_sino, h_img), e2e_steps, stream)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    # ---- the same batch with FP16-stored pairs (the precision variant; its
    # own tuned plan): the whole step and its backprojection launch alone
    fp16 = None
    if world == 1 and not args.no_configs:
        plan16 = fbp.Plan(spec0.n_pix, spec0.n_angles, spec0.n_det, filter=spec0.filter,
                          autotune=True, batch_hint=min(S, 64), q_storage=2)
        works16 = [plan16.empty_workspace() for _ in range(S)]
        full16 = fbp.Batch([plan16] * S, sinos, images, works16)
        bp16 = fbp.Batch([plan16] * S, sinos, images, works16, parts=fbp.FBP_BATCH_BACKPROJECT)
        full16.launch()
        ms16 = _timed(full16.launch, max(args.steps // 2, 5), stream) / max(args.steps // 2, 5)
        bp16.launch()
        _, bp16_ms = _timed(bp16.launch, max(args.steps // 4, 5), stream, per_launch=True)
        full16.status()
        t16 = plan16.tuning or {}
        fp16 = {"slices_per_s": S / (ms16 / 1e3), "ms_per_step": ms16,
                "backprojection_gupdates_per_s":
                    S * spec0.updates / (sum(bp16_ms) / len(bp16_ms) / 1e3) / 1e9,
                "tile": [t16.get("tile_x"), t16.get("tile_y"), t16.get("angle_chunk")],
                "what": "the headline batch with (mid, slope) pairs stored in FP16 and "
                        "summed in FP32 (mixed-precision FMA); error stated, no bar"}
        full16.close()
        bp16.close()
        del works16

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
    achieved = S * upd / (bp_mean / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "gupdates_per_s": value * upd / 1e9,
        "plain_path": {"value": S * plain_steps / (plain_ms / 1e3), "unit": "slices/s",
                       "what": "one fbp_reconstruct call per slice, same slices and stream"},
        "filter_ms_per_step": filt_ms,
        "fp16_pairs_batched": fp16,
        "config": {"workload": WORKLOAD_NAME, "slices_per_step": S * world,
                   "path": ("batched: one captured graph per step (%s + one persistent "
                            "backprojection launch over all slices' tiles)" %
                            ("per-slice direct filter launches" if plan.filter_path == 3 else
                             "one %s filter launch over all slices' rows" %
                             ROUTE_NAMES[plan.filter_path])),
                   "l2": f"inputs larger than L2: {resident_mb:.0f} MB resident per GPU",
                   "tuned": {k: plan.tuning[k] for k in ("filter_path", "fft_len", "tile_x",
                                                         "tile_y", "angle_chunk")},
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "bp_persistent_kernel", "achieved": achieved,
                     "peak": peak_gups, "unit": "Gupdates/s", "frac": achieved / peak_gups,
                     "traffic": BP_TRAFFIC.get((f"{spec0.n_pix}x{spec0.n_angles}x{spec0.n_det}",
                                                S, plan.tuning["tile_x"], plan.tuning["tile_y"],
                                                plan.tuning["angle_chunk"])),
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                     "smem_ceiling": {
                         "gupdates_per_s": SMEM_UPDATES_PER_CLK_SM * sms * sm_mhz / 1e3,
                         "frac": achieved / (SMEM_UPDATES_PER_CLK_SM * sms * sm_mhz / 1e3),
                         "basis": "one 8-byte pair per update; an 8-byte warp load is two "
                                  "128-byte shared-memory wavefronts: 16 updates/clk/SM"},
                     "peak_basis": f"{FP32_LANES_PER_SM} FP32 lanes x {sms} SMs x {sm_mhz:.0f} "
                                   f"MHz ({pk_kind} sm_max_mhz) / {OPS_PER_UPDATE} FP32 ops per "
                                   f"update",
                     "launch_ms": bp_mean, "updates_per_launch": S * upd},
        "e2e": {"value": S * e2e_steps * world / (e2e_ms / 1e3), "unit": "slices/s",
                "h2d_bytes_per_step": S * spec0.n_angles * spec0.n_det * 4,
                "d2h_bytes_per_step": S * spec0.n_pix ** 2 * 4},
        "gpu_launches": full.kernel_count * args.steps,
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
        # the paper's sequential CPU arm: the same slice on one host core
        t1 = cpu_fbp_time([spec0], sample, 1)
        line["cpu_one_core"] = {"value": 1.0 / t1, "unit": "slices/s", "cores": 1,
                                "kind": "oracle", "sample": "the same slice on one host core"}
    for b in (full, bp_only, filt_only):
        b.close()
    if serve_result is not None:
        line["serving"] = serve_result
    if world == 1 and not args.no_uneven:
        line["batched_uneven"] = run_uneven(fbp)
    if world == 1 and not args.no_configs:
        line["configs"] = run_configs(fbp)
    if "cpu_baseline" in line and not args.no_configs:
        # last: tens of seconds on every host core, which also disturbed the
        # serving loop's latency when it ran just before it
        line["cpu_baseline"]["configs"] = cpu_config_times(os.cpu_count() or 1)
    if serve_sample:
        line["serving"]["oracle_check"] = check_serving_sample(serve_sample,
                                                               os.cpu_count() or 1)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--slices", type=int, default=64)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the 64-uneven-slice batch measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-configuration measurements")
    ap.add_argument("--filter-path", choices=sorted(FILTER_PATHS), default="auto",
                    help="ramp-filter route (auto: the autotuner picks)")
    ap.add_argument("--tile", default="",
                    help="backprojection tile WxH (32x64, 32x32, 8x32) instead of the tuned one")
    ap.add_argument("--chunk", type=int, default=16, choices=(8, 16, 32),
                    help="angles per shared-memory stage with --tile")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson serving run (0 = skip)")
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

#!/usr/bin/env python
"""FBP throughput at 2048^3 on GB300: GVoxel/s of chunked parallel-beam FBP
(dark/flat normalisation with -log, Shepp-Logan ramp filter, LineRec
backprojection) from 2048 uint16 projections of 2048 x 2048 pixels.

One step = one full reconstruction of the 2048^3 volume, every slice chunk
through normalise+filter and backprojection.  `value` is measured with the
uint16 projections already in HBM; `e2e` through the same C-ABI call with
page-locked HOST input and output buffers (host->device copies of the raw
slabs and device->host copies of the volume inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) each rank reconstructs its own seeded dataset (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FBP GVoxel/s at 2048^3 (FP16 vs FP32, at stated L2 error); % of roofline"
# Paper, Table 2: LineRec (this method), FP32, N = 2048, 80 s on one A100 incl. I/O.
PAPER_LINEREC_GVOXS = 2048 ** 3 / 80.0 / 1e9
DATA = ("synthetic: seeded porous-medium phantom (spheres r = 3-40 px, density 0.2-1.0, 40 % solid in a "
        "0.45 N cylinder), exact line integrals, Poisson uint16 frames I0 = 3e4 with 20 dark / 20 flat frames")


# ----------------------------------------------------------- multi-rank --

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a scalar over ranks (identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device_index=None):
    if world > 1:
        import torch.distributed as dist
        if device_index is None:
            dist.barrier()
        else:
            dist.barrier(device_ids=[device_index])


def slab(nz: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous z-slab [z0, z1) of rank among world (the paper's start/end rows)."""
    from paper_2209_08450_gb300.slabs import slab as _slab
    return _slab(nz, rank, world)


# ---------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU leg --

def oracle_fbp_slices(raw, dark, flat, theta, center, n_threads=None):
    """FP64 oracle FBP of a few slices (normalise, filter, backproject)."""
    import oracle
    p = oracle.normalize(raw, oracle.frame_mean(dark), oracle.frame_mean(flat))
    q = oracle.filter_sino(p, center, "shepp", "edge")
    return oracle.backproject(q, theta, raw.shape[-1] / 2.0, raw.shape[-1])


def host_sample(n: int, ntheta: int, slices, seed: int = 0):
    """Host copy of a few slices of the porous workload (torch on the CPU)."""
    import numpy as np
    import synth.gpu as sgpu
    raw, dark, flat, theta, center, mu = sgpu.porous_frames(n, ntheta, n, seed=seed, device="cpu",
                                                            slices=np.asarray(slices))
    u = lambda t: t.numpy().view(np.uint16)
    return u(raw), u(dark), u(flat), theta, center


def cpu_baseline(n: int, ntheta: int, nslices: int) -> dict:
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    raw, dark, flat, theta, center = host_sample(n, ntheta, list(range(n // 2, n // 2 + nslices)))
    t0 = time.perf_counter()
    oracle_fbp_slices(raw, dark, flat, theta, center)
    dt = time.perf_counter() - t0
    return {"value": nslices * n * n / dt / 1e9, "unit": "GVoxel/s", "cores": cores, "kind": "oracle",
            "sample": "%d slices of the %d^3 workload (%d angles): FP64 normalise + numpy-FFT filter + C/OpenMP "
                      "LineRec backprojection, %.1f s" % (nslices, n, ntheta, dt), "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n, nt = args.size, args.size
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    oracle.build()
    nsl = args.ref_slices
    raw, dark, flat, theta, center = host_sample(n, nt, list(range(n // 2, n // 2 + nsl)))
    for _ in range(args.warmup):
        oracle_fbp_slices(raw, dark, flat, theta, center)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_fbp_slices(raw, dark, flat, theta, center)
    dt = (time.perf_counter() - t0) / args.steps
    v = nsl * n * n / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GVoxel/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": v / PAPER_LINEREC_GVOXS, "dtype": "f64", "data": DATA,
        "config": {"workload": "%d slices of the %d^3 FBP workload (%d angles) per step" % (nsl, n, nt),
                   "n": n, "ntheta": nt, "l2": "host run"},
        "cpu_baseline": {"value": v, "unit": "GVoxel/s", "cores": cores, "kind": "oracle",
                         "sample": "%d slices per step, FP64 oracle on the host cores" % nsl},
        "e2e": {"value": v, "unit": "GVoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------- other hot-path rows --

def _peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Reconstruction paths: volume dtype, sinogram storage (None: the library's
# choice), default chunk.  "f32" is FP32 volumes from FP16 hi/lo sinogram pairs
# (tensor cores, FP32-accurate), "f32_cuda" FP32 sinograms on the CUDA cores.
PATHS = {
    "f32": ("float32", None, 256),
    "f16": ("float16", None, 256),
    "bf16": ("bfloat16", None, 256),
    "f32_cuda": ("float32", "float32", 32),
    "f32_frec": ("float32", "float32", 64),
    "f16_frec": ("float16", "float16", 64),
}
# Paths reconstructed by FourierRec (Fourier-slice gridding) instead of LineRec.
FOURIERREC = {"f32_frec": 7, "f16_frec": 5}  # path -> window width


# DRAM bytes (read + write) per backprojector launch from ncu captures of these
# exact launch shapes (slices, angles, n) -> bytes, file under profiles/.  Set
# an entry to None when its kernel changes.
PROFILED_TRAFFIC = {
    "f32": ((256, 2048, 2048), 396.80e9 + 4.30e9, "profiles/k_backproject_tc_split_f32_2048sq_256slices.md"),
    "f16": ((256, 2048, 2048), 158.44e9 + 2.14e9, "profiles/k_backproject_tc_f16_2048sq_256slices.md"),
}


def _traffic(path, nz, nt, n):
    e = PROFILED_TRAFFIC.get(path)
    if e and e[0] == (nz, nt, n):
        return e[1], e[2]
    return None, None


def bp_roofline(tcp, dev, path, nz, nt, n, ms) -> dict:
    """Roofline of the backprojector launch of this path and chunk.

    LineRec's work is the interpolation count nz * n^2 * ntheta, each 2 FP32
    operations (the lerp as an FMA and the accumulation), so its ceiling is
    the FP32 FMA rate: SMs x 128 lanes x clock / 2 interpolations per second.
    `frac` is always interpolations/s against that ceiling, whichever kernel
    runs.  Alongside: the shared-memory roof of the CUDA-core kernel (per 32
    interpolations a warp needs 2 wavefronts for FP32 samples or 1 for 16-bit
    sample pairs: 16 or 32 interpolations per clock per SM), and for the
    tensor-core kernel the dense MMA utilisation it reaches (each
    interpolation is one entry of a dense 128 x 32 x N product, 64 flops, 30
    of the 32 weights in a row zero; three products in split mode) against the
    measured bf16 peak, a diagnostic of the tensor pipe, not of the method."""
    import torch
    pk = _peaks()
    clk_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    interps = nz * n * n * nt
    if path in FOURIERREC:
        # gridding work: every polar sample (ntheta x (M + 1) per slice pair)
        # reaches W x W grid nodes with one complex-by-real multiply-add
        # (4 flops); against the FP32 FMA peak of the CUDA cores
        w = FOURIERREC[path]
        m = 1
        while m < 2 * n:
            m *= 2
        flops = ((nz + 1) // 2) * nt * (m + 1) * w * w * 4
        peak = sms * 128 * 2 * clk_max * 1e6
        ach = flops / (ms * 1e-3)
        return {"bound": "alu", "kernel": "tcp_fourierrec (row FFT, gather, column and row inverse FFTs; "
                                          "k_frec_gather is the dominant kernel)",
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "ms_per_launch": ms, "window_width": w,
                "peak_basis": "FP32 FMA lanes: %d SMs x 128 x 2 flops x %.0f MHz (max SM clock); the time is the "
                              "whole backprojector call, not the gather kernel alone" % (sms, clk_max)}
    vdt, sdt, _ = PATHS[path]
    split = path == "f32"
    fma_ceiling = sms * 128 * clk_max * 1e6 / 2
    ach = interps / (ms * 1e-3)
    traffic, tsrc = _traffic(path, nz, nt, n)
    sd = "f16x2" if split else getattr(torch, sdt or vdt)
    kernel = tcp.get_backproject_config(nz, nt, n, n, sd, getattr(torch, vdt))[3]
    # shared-memory roof: 8 B per interpolation for FP32 samples (16 interp/clk),
    # 4 B for 16-bit sample pairs and for the FP32 slice-pair form with its
    # sample reuse (32 interp/clk)
    per_clk = 16 if (sdt or vdt) == "float32" and kernel != 2 else 32
    smem_roof = sms * per_clk * clk_max * 1e6
    out = {"bound": "alu", "achieved": ach / 1e9, "peak": fma_ceiling / 1e9, "unit": "Ginterp/s",
           "frac": ach / fma_ceiling, "traffic": traffic, "traffic_source": tsrc, "ms_per_launch": ms,
           "interps_per_launch": interps, "algorithmic_bytes_per_launch": None,
           "kernel_only_gvoxel_s": nz * n * n / (ms * 1e-3) / 1e9,
           "peak_basis": "FP32 FMA ceiling of LineRec: %d SMs x 128 FP32 lanes x %.0f MHz (max SM clock) / 2 "
                         "operations per interpolation (derived from the lane count and clock; no measured FP32 "
                         "peak exists)" % (sms, clk_max)}
    # algorithmic HBM bytes: the sinogram chunk read once, the volume written once
    sbytes = (4 if split else (4 if (sdt or vdt) == "float32" else 2)) * nz * nt * n
    vbytes = {"float32": 4, "float16": 2, "bfloat16": 2}[vdt] * nz * n * n
    out["algorithmic_bytes_per_launch"] = sbytes + vbytes
    if kernel in (1, 3):
        fl = 192 if split else 64
        bpk = float(pk.get("bf16_tflops", 1900.0))
        mma = interps * fl / (ms * 1e-3) / 1e12
        out.update({"kernel": "k_backproject_tc (LineRec on tcgen05.mma, %s)" %
                              ("FP16 hi/lo pairs, 3 products" if split else path),
                    "mma_tflops_executed": mma, "mma_frac_of_bf16_peak": mma / bpk,
                    "mma_basis": "%d dense MMA flops per interpolation against the measured dense bf16 burst "
                                 "(MEASURED_PEAKS.json, of measured); 30 of the 32 weights in each operand row are "
                                 "zero" % fl})
    else:
        out.update({"kernel": "k_backproject (LineRec, %s storage%s)" % (
                        sdt or vdt, ", FP32 slice pairs, packed FMAs, sample reuse down columns" if kernel == 2 else ""),
                    "smem_roof_ginterp_s": smem_roof / 1e9, "frac_of_smem_roof": ach / smem_roof,
                    "smem_basis": "shared-memory pipe: %d SMs x %d interp/clk x %.0f MHz" % (sms, per_clk, clk_max)})
    return out


def pipeline_trace(tcp, raw_h, dark_h, flat_h, theta, center, vol_h, chunk, sdt) -> dict:
    """One traced run of the host-buffer pipeline through a plan: per chunk the
    upload, compute and download intervals (CUDA events), and how much of the
    copy time overlaps compute of another chunk."""
    nz, n = vol_h.shape[0], vol_h.shape[1]
    plan = tcp.Plan(theta, raw_h.shape[2], nz, center, n=n, dtype=vol_h.dtype, chunk_nz=chunk, sino_dtype=sdt,
                    host_raw=True, host_vol=True, host_frames=max(dark_h.shape[0], flat_h.shape[0]), trace=True)
    try:
        plan.fbp(raw_h, dark_h, flat_h, out=vol_h)
        t = plan.trace()
    finally:
        plan.close()
    comp = [(r[2], r[3]) for r in t]

    def hidden(a, b):  # part of [a, b] covered by compute intervals
        return sum(max(0.0, min(b, c1) - max(a, c0)) for c0, c1 in comp)

    up = [(r[0], r[1]) for r in t if r[0] >= 0]
    down = [(r[4], r[5]) for r in t if r[4] >= 0]
    up_ms = sum(b - a for a, b in up)
    down_ms = sum(b - a for a, b in down)
    return {"chunks": int(t.shape[0]), "total_ms": float(t[:, :].max()),
            "compute_ms": float(sum(b - a for a, b in comp)),
            "upload_ms": up_ms, "upload_hidden_frac": sum(hidden(a, b) for a, b in up) / max(up_ms, 1e-9),
            "download_ms": down_ms, "download_hidden_frac": sum(hidden(a, b) for a, b in down) / max(down_ms, 1e-9),
            "per_chunk_ms": [[round(float(x), 3) for x in r] for r in t]}


def lprec_step2_fma(n: int, nt: int, os: float = 2.0) -> float:
    """Multiply-adds of LpRec's span convolution (its dominant step) per slice:
    4 per (log-polar grid point, angle of the span), three spans; grid sizes
    as the library sets them (log-polar origin at 4 R, steps 1/os pixel at the
    far radius, 12-point margins)."""
    import math
    R = n / math.sqrt(2.0) + 2.0
    a = 4.0 * R
    drho = 1.0 / (os * (a + R))
    dth = math.pi / nt
    p = math.ceil(os * (a + R) * dth)
    dpsi = dth / p
    nrho = math.ceil((math.log(a + R) - math.log(a - R)) / drho) + 25
    npsi = 2 * math.ceil((math.asin(R / a) + 12 * dpsi) / dpsi) + 1
    return 4.0 * nrho * npsi * nt


def measure_lprec(tcp, raw, dark, flat, theta, center, n, nslices, steps=2) -> dict:
    """LpRec FBP (oversampling 2) of `nslices` middle slices of the resident
    stack (views, no copy): GVox/s, the span convolution's FMA rate against
    the FP32 FMA ceiling, and the distance to the direct cubic-spline sums on
    sampled voxels of one slice (the quantity LpRec approximates)."""
    import numpy as np
    import torch
    import oracle
    from oracle import lprec as olp
    nz = raw.shape[1]
    z0 = max(0, nz // 2 - nslices // 2)
    z1 = min(nz, z0 + nslices)
    r, d, f = raw[:, z0:z1], dark[:, z0:z1], flat[:, z0:z1]
    vol = torch.empty((z1 - z0, n, n), dtype=torch.float32, device=raw.device)

    def step():
        tcp.fbp(r, d, f, theta, center, out=vol, algorithm="lprec")
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pk = _peaks()
    sms = torch.cuda.get_device_properties(raw.device).multi_processor_count
    fma_peak = sms * 128 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    fma = lprec_step2_fma(n, len(theta)) * (z1 - z0)
    zc = (z1 - z0) // 2
    rr = r[:, zc:zc + 1].cpu().numpy().view(np.uint16)
    p = oracle.normalize(rr, oracle.frame_mean(d[:, zc:zc + 1].cpu().numpy().view(np.uint16)),
                         oracle.frame_mean(f[:, zc:zc + 1].cpu().numpy().view(np.uint16)))
    q = oracle.filter_sino(p, center, "shepp")[0]
    rng = np.random.default_rng(2)
    ix, iy = rng.integers(0, n, 200), rng.integers(0, n, 200)
    ref = olp.backproject_spline_points(q, theta, n / 2.0, n, ix, iy)
    got = vol[zc].double().cpu().numpy()[iy, ix]
    return {"workload": "%d middle slices of the %d^3 workload, %d angles, LpRec FBP (oversampling 2), FP32"
                        % (z1 - z0, n, len(theta)),
            "ms_per_step": ms, "value": (z1 - z0) * n * n / (ms * 1e-3) / 1e9, "unit": "GVoxel/s",
            "roofline": {"bound": "alu", "kernel": "k_lp_span (span convolution; whole call timed)",
                         "achieved": fma / (ms * 1e-3) / 1e12, "peak": fma_peak / 1e12, "unit": "TFMA/s",
                         "frac": fma / (ms * 1e-3) / fma_peak, "traffic": None,
                         "peak_basis": "%d SMs x 128 FP32 lanes x max SM clock; 4 multiply-adds per (log-polar "
                                       "grid point, angle)" % sms},
            "rel_l2_vs_cubic_spline_sums": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}


def measure_rows(dev) -> dict:
    """Differentiable least-squares pair (512 x 512 x 64, 720 angles, 512-pixel
    detector) and the uneven batch (6 stacks, one persistent graph replay)."""
    import numpy as np
    import torch

    import synth
    import synth.gpu as sgpu
    import paper_2209_08450_gb300 as tcp
    from paper_2209_08450_gb300 import autograd as ag
    from paper_2209_08450_gb300.batch import Batch

    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    # LineRec's ceiling (interpolations/s), as in bp_roofline: FP32 lanes x max clock / 2
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma_ceiling = sms * 128 * float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 2
    # a7: gradient descent on ||P x - y||^2 through the autograd pair
    n, nz, nt = 512, 64, 720
    theta = synth.uniform_theta(nt)
    ells = synth.random_ellipsoids(np.random.default_rng(4), 64, n, float(nz))
    x_true = sgpu.rasterize_ellipsoids(ells, n, np.arange(nz) + 0.5 - nz / 2.0, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    y = tcp.project(x_true, theta, n / 2.0, ndet=n)
    y = y + 1e-2 * torch.randn(y.shape, generator=g, device=dev)
    # untimed warm-up solve: first-use costs (module loading, table builds) stay
    # outside the timed 50 iterations
    ag.lsq_gradient_descent(y, theta, n / 2.0, n, iters=2)
    torch.cuda.synchronize()
    losses = []
    t0 = time.perf_counter()
    ag.lsq_gradient_descent(y, theta, n / 2.0, n, iters=50, callback=lambda i, l: losses.append(l))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    x = torch.zeros_like(x_true)
    pj = ev_time(lambda: tcp.project(x_true, theta, n / 2.0, out=y), 3)
    bj = ev_time(lambda: tcp.backproject(y, theta, n / 2.0, out=x), 3)
    interps = nz * n * n * nt
    out["a7_least_squares"] = {
        "workload": "512x512x64 ellipsoids, 720 angles, 512-pixel detector, sigma 1e-2, 50 GD iterations (operator-norm estimate included) after an untimed 2-iteration warm-up solve",
        "seconds_50_iterations": wall, "loss_ratio_50": losses[-1] / losses[0],
        "project_ms": pj, "backproject_ms": bj, "project_ginterp_s": interps / pj / 1e6,
        "backproject_ginterp_s": interps / bj / 1e6,
        "project_frac_of_fma_ceiling": interps / (pj * 1e-3) / fma_ceiling,
        "backproject_frac_of_fma_ceiling": interps / (bj * 1e-3) / fma_ceiling}
    del x_true, y, x
    # a8: six uneven stacks, FP16 storage, one graph replay
    widths = (512, 768, 1024, 1536, 2048, 2560)
    angles = (400, 900, 1200, 1800, 2048, 3000)
    ds = []
    for i, (w, a) in enumerate(zip(widths, angles)):
        raw, dark, flat, th, c, mu = sgpu.ellipsoid_frames(w, a, 32, seed=10 + i, device=dev, count=24)
        ds.append(dict(raw=raw, dark=dark, flat=flat, theta=th, center=c,
                       vol=torch.empty((32, w, w), dtype=torch.float32, device=dev)))
    b = Batch(ds, sino_dtype=torch.float16, autotune=True)
    st = torch.cuda.Stream()
    b.capture(st)
    torch.cuda.synchronize()

    def replay():
        b.replay(st)
    replay()
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(3):
        replay()
    e1.record(st)
    st.synchronize()
    ms = e0.elapsed_time(e1) / 3
    vox = sum(32 * w * w for w in widths)
    interps = sum(32 * w * w * a for w, a in zip(widths, angles))
    info = b.info()
    out["a8_uneven_batch"] = {
        "workload": "6 stacks x 32 slices, widths 512-2560, 400-3000 angles, FP16 sinograms, one graph replay",
        "ms_per_replay": ms, "gvoxel_s": vox / ms / 1e6, "ginterp_s": interps / ms / 1e6,
        "frac_of_fma_ceiling": interps / (ms * 1e-3) / fma_ceiling,
        "config": info["config"], "kernel": info["kernel"], "tuned_ms": info["tuned_ms"],
        "grid_blocks": info["grid_blocks"],
        "work_units": info["work_units"]}
    b.close()
    del ds
    # f2: multi-centre "try" reconstruction of one 2048^2 slice, 64 candidate axes
    raw, dark, flat, th, c, mu = sgpu.porous_frames(2048, 2048, 2048, seed=3, device=dev, slices=np.array([1024]))
    centers = c + 0.25 * (np.arange(64) - 32)
    vol = torch.empty((64, 2048, 2048), dtype=torch.float32, device=dev)
    tms = ev_time(lambda: tcp.try_centers(raw, dark, flat, th, centers, slice=0, out=vol), 3)
    fms = ev_time(lambda: tcp.try_centers(raw, dark, flat, th, centers, slice=0, out=vol, algorithm="fourierrec"), 3)
    out["f2_try_centers"] = {
        "workload": "one 2048^2 slice of the porous workload, 2048 angles, 64 candidate centres (step 0.25 px), "
                    "FP32 volume (LineRec: from FP16 hi/lo pairs; FourierRec: FP32 rows, window 7)",
        "ms": tms, "gvoxel_s": 64 * 2048 * 2048 / tms / 1e6,
        "fourierrec_ms": fms, "fourierrec_gvoxel_s": 64 * 2048 * 2048 / fms / 1e6}
    del raw, dark, flat, vol
    return out


# ------------------------------------------------------------- GPU leg --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--nz", type=int, default=0, help="slices (default: size); a small case of the same launches")
    ap.add_argument("--dtype", default="f32", choices=list(PATHS),
                    help="headline path (f32: FP32 volume from FP16 hi/lo sinogram pairs on the tensor cores; "
                         "*_frec: FourierRec)")
    ap.add_argument("--chunk", type=int, default=0, help="slices per chunk (0: the path's default)")
    ap.add_argument("--variants", default="f32,f16,bf16,f32_cuda,f32_frec,f16_frec")
    ap.add_argument("--variant-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-slices", type=int, default=16)
    ap.add_argument("--ref-slices", type=int, default=1)
    ap.add_argument("--lprec-slices", type=int, default=32, help="slices of the LpRec variant (0: skip)")
    ap.add_argument("--parity-slices", type=int, default=2)
    ap.add_argument("--no-rows", action="store_true", help="skip the least-squares and batch rows")
    ap.add_argument("--split", default="replicas", choices=["replicas", "slab"],
                    help="N > 1: 'replicas' (each rank its own seeded dataset, weak scaling) or 'slab' (one dataset, "
                         "rank r reconstructs its z-slab through views of the shared stack, strong scaling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2209_08450_gb300 as tcp
    import synth.gpu as sgpu

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = nt = args.size

    # ---- input: seeded synthetic dataset, resident in HBM (not timed)
    t_gen = time.perf_counter()
    nz = args.nz or n
    split = args.split == "slab" and world > 1
    raw, dark, flat, theta, center, mu = sgpu.porous_frames(n, nt, n, seed=0 if split else rank, device=dev,
                                                            slices=np.arange((n - nz) // 2, (n - nz) // 2 + nz))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    raw_bytes = raw.numel() * 2
    def vdt_of(path):
        return getattr(torch, PATHS[path][0])

    def sdt_of(path):
        return None if PATHS[path][1] is None else getattr(torch, PATHS[path][1])

    def chunk_for(path):
        return args.chunk or PATHS[path][2]
    hp = args.dtype
    hdt = vdt_of(hp)
    nchunks = (nz + chunk_for(hp) - 1) // chunk_for(hp)

    from paper_2209_08450_gb300 import slabs
    z0_r, z1_r = slabs.slab(nz, rank, world) if split else (0, nz)
    my_nz = z1_r - z0_r  # slices this rank reconstructs

    def run_steps(path, steps, warmup, out):
        stream = torch.cuda.current_stream()
        # split mode: this rank's z-slab of the one dataset, through views
        fbp = (lambda r, d, f, th, c, **kw: slabs.reconstruct_slab(r, d, f, th, c, kw.pop("out"), rank, world, **kw)) \
            if split else tcp.fbp

        def step():
            fbp(raw, dark, flat, theta, center, out=out, chunk_nz=chunk_for(path), sino_dtype=sdt_of(path),
                    algorithm="fourierrec" if path in FOURIERREC else "linerec", width=FOURIERREC.get(path, 0),
                    stream=stream)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        barrier(world, local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world, local)
        return reduce_max(e0.elapsed_time(e1) / steps, world, dev)

    # ---- headline: FP32 storage and arithmetic (unless --dtype says otherwise)
    vol = torch.empty((my_nz, n, n), dtype=hdt, device=dev)
    with ClockSampler(local) as clk:
        ms = run_steps(hp, args.steps, args.warmup, vol)
    clocks = clk.summary()
    # replicas: every rank a full dataset; slab: the ranks share one
    value = (nz if split else world * nz) * n * n / (ms * 1e-3) / 1e9

    # ---- parity on sampled slices (oracle on the same uint16 frames)
    def parity(v, zs, path=None):
        import oracle
        from oracle import fourierrec as frc
        rng = np.random.default_rng(1)
        errs = []
        frec = path in FOURIERREC
        npts = 24 if frec else 2000  # the exact FourierRec sums cost ntheta x 2 ndet per voxel
        for z in zs:
            r = raw[:, z:z + 1].cpu().numpy().view(np.uint16)
            d = dark[:, z:z + 1].cpu().numpy().view(np.uint16)
            f = flat[:, z:z + 1].cpu().numpy().view(np.uint16)
            p = oracle.normalize(r, oracle.frame_mean(d), oracle.frame_mean(f))
            q = oracle.filter_sino(p, center, "shepp")[0]
            ix, iy = rng.integers(0, n, npts), rng.integers(0, n, npts)
            if frec:
                ref = frc.backproject_exact_points(q, theta, n / 2.0, n, ix, iy)
            else:
                ref = oracle.backproject_points(q, theta, n / 2.0, n, ix, iy)
            got = v[z].double().cpu().numpy()[iy, ix]
            errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        return float(max(errs))

    zs = [int(x) for x in np.linspace(nz // 5, 4 * nz // 5, args.parity_slices)]
    if split:  # rank 0 checks slices of its own slab (vol holds only that slab)
        zs = [int(x) for x in np.linspace(my_nz // 5, 4 * my_nz // 5, args.parity_slices)] if my_nz > 0 else []
    par = {args.dtype: parity(vol, zs, hp)} if rank == 0 and zs else {}

    # ---- dominant kernel, timed alone on one filtered chunk (same launch shape)
    dm, fm = tcp.frame_mean(dark), tcp.frame_mean(flat)

    def time_kernel(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def path_kernels(path, out_vol):
        """(backprojector ms, fused normalise+filter ms, filter bytes) on one
        chunk, with the sinogram in the form the path's pipeline stores."""
        c = min(chunk_for(path), nz)
        zc = max(0, nz // 2 - c)
        vdt, sdt = vdt_of(path), sdt_of(path)
        if sdt is None:  # scaled storage: ramp x 2^10, pi/ntheta/2^10 at the voxel store
            sd = "f16x2" if vdt == torch.float32 else vdt
            w, sc = 1024.0, np.pi / nt / 1024.0
        else:
            sd, w, sc = sdt, None, 1.0
        nf = lambda: tcp.normalize_filter(raw[:, zc:zc + c], dm[zc:zc + c], fm[zc:zc + c], center, dtype=sd,
                                          weight=w)
        sino = nf()
        if path in FOURIERREC:
            ms_bp = time_kernel(lambda: tcp.fourierrec(sino, theta, n / 2.0, out=out_vol[:c], scale=sc,
                                                       width=FOURIERREC[path]))
        else:
            ms_bp = time_kernel(lambda: tcp.backproject(sino, theta, n / 2.0, out=out_vol[:c], scale=sc))
        holder = {}

        def nf_into():
            holder["s"] = tcp.normalize_filter(raw[:, zc:zc + c], dm[zc:zc + c], fm[zc:zc + c], center,
                                               out=sino, weight=w)
        ms_nf = time_kernel(nf_into)
        nbytes = nt * c * n * 2 + sino.numel() * sino.element_size()
        del sino, holder
        return c, ms_bp, ms_nf, nbytes

    kc, bp_ms, nf_ms, nf_bytes = path_kernels(hp, vol)
    interps = kc * n * n * nt
    roofline = bp_roofline(tcp, dev, hp, kc, nt, n, bp_ms)
    hbm = float(_peaks().get("hbm_gbs", 6800.0))  # the profiling recipe's fallback when no measurement exists
    secondary = {"normalize_filter": {"bound": "hbm", "achieved": nf_bytes / (nf_ms * 1e-3) / 1e9, "peak": hbm,
                                      "unit": "GB/s", "frac": nf_bytes / (nf_ms * 1e-3) / 1e9 / hbm,
                                      "ms_per_launch": nf_ms}}

    # ---- other paths: 16-bit storage, FP32 sinograms on the CUDA cores
    variants = {}
    for name in [v for v in args.variants.split(",") if v and v != hp and not split]:
        vv = torch.empty((nz, n, n), dtype=vdt_of(name), device=dev)
        vms = run_steps(name, args.variant_steps, 1, vv)
        variants[name] = {"value": world * nz * n * n / (vms * 1e-3) / 1e9, "ms_per_step": vms,
                          "speedup_vs_headline": ms / vms, "chunk_nz": chunk_for(name),
                          "sino_storage": "f16x2" if name == "f32" else (PATHS[name][1] or PATHS[name][0]),
                          "algorithm": "fourierrec (window %d)" % FOURIERREC[name] if name in FOURIERREC
                          else "linerec"}
        vc, vms_k, _, _ = path_kernels(name, vv)
        variants[name]["roofline"] = bp_roofline(tcp, dev, name, vc, nt, n, vms_k)
        if rank == 0 and zs:
            variants[name]["rel_l2_vs_fp64_oracle"] = parity(vv, zs, name)
        del vv

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e and not split:
        del vol
        torch.cuda.empty_cache()
        raw_h = torch.empty(raw.shape, dtype=raw.dtype, pin_memory=True)
        raw_h.copy_(raw)
        dark_h = dark.cpu().pin_memory()
        flat_h = flat.cpu().pin_memory()
        vol_h = torch.empty((nz, n, n), dtype=hdt, pin_memory=True)
        stream = torch.cuda.current_stream()

        def e2e_step():
            tcp.fbp(raw_h, dark_h, flat_h, theta, center, out=vol_h, chunk_nz=chunk_for(hp), sino_dtype=sdt_of(hp),
                    algorithm="fourierrec" if hp in FOURIERREC else "linerec", width=FOURIERREC.get(hp, 0),
                    stream=stream)
        e2e_step()
        torch.cuda.synchronize()
        barrier(world, local)
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / args.steps * 1e3
        barrier(world, local)
        ems = reduce_max(max(e0.elapsed_time(e1) / args.steps, wall), world, dev)
        e2e = {"value": world * nz * n * n / (ems * 1e-3) / 1e9, "unit": "GVoxel/s", "ms_per_step": ems,
               "h2d_bytes_per_step": raw_h.numel() * 2 + dark_h.numel() * 2 + flat_h.numel() * 2,
               "d2h_bytes_per_step": vol_h.numel() * vol_h.element_size()}
        if rank == 0 and zs:
            par[args.dtype + "_e2e"] = parity(vol_h, zs[:1], hp)
            par[args.dtype + "_e2e_slices"] = parity(vol_h, zs, hp)
        # per-chunk timeline of one more run (untimed, through a plan with the
        # same options): how much of the copy time hides under compute
        if rank == 0 and hp not in FOURIERREC:
            e2e["pipeline_trace"] = pipeline_trace(tcp, raw_h, dark_h, flat_h, theta, center, vol_h, chunk_for(hp),
                                                   sdt_of(hp))
        del raw_h, vol_h

    if args.lprec_slices > 0 and not split:
        variants["f32_lprec"] = measure_lprec(tcp, raw, dark, flat, theta, center, n, min(args.lprec_slices, nz))

    rows = None
    if not args.no_rows and world == 1 and not split:
        del raw, dark, flat
        torch.cuda.empty_cache()
        rows = measure_rows(dev)
    cpu = cpu_baseline(n, nt, args.cpu_slices) if rank == 0 and world == 1 and args.cpu_slices > 0 else None
    if rank == 0:
        if hp in FOURIERREC:
            # per chunk: normalise+filter, the angle/phase table kernel, and per
            # batch of slice pairs: row FFT, gather, column and row inverse FFTs
            m = l = 1
            while m < 2 * n:
                m *= 2
            while l < 2 * n:
                l *= 2
            per_pair = 8 * (nt * (m + 1) + n * l + l * l)
            cz = min(chunk_for(hp), nz)
            nb = max(1, min((cz + 1) // 2, (3 << 29) // per_pair))
            per_chunk = [2 + 4 * (((min(cz, nz - z0) + 1) // 2 + nb - 1) // nb) for z0 in range(0, nz, cz)]
            launches_per_step = 2 + sum(per_chunk)
        else:
            launches_per_step = 2 + 2 * nchunks  # 2 frame means + per chunk: normalise+filter, backproject
        out = {
            "metric": METRIC, "value": value, "unit": "GVoxel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong" if split else "weak",
            "vs_baseline": value / PAPER_LINEREC_GVOXS, "dtype": "f32" if hp.startswith("f32") else hp,
            "path": hp, "data": DATA,
            "config": {"workload": "%dx%d^2 FBP (%s) from %d uint16 projections of %dx%d, angles on [0, pi), "
                                   "Shepp-Logan filter, %d-slice chunks, inputs resident in HBM"
                                   % (nz, n, "FourierRec, window %d" % FOURIERREC[hp] if hp in FOURIERREC else "LineRec",
                                      nt, n, nz, chunk_for(hp)),
                       "n": n, "nz": nz, "ntheta": nt, "chunk_nz": chunk_for(hp),
                       "sino_storage": "f16x2" if hp == "f32" else (PATHS[hp][1] or PATHS[hp][0]),
                       "l2": "inputs larger than L2 (%.1f GB uint16 per step)" % (raw_bytes / 1e9),
                       "parallelism": ("z-slab split of one dataset over %d ranks, no collective on the data path"
                                       % world) if split else ("%d independent replicas" % world)},
            "roofline": roofline, "secondary_kernels": secondary, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
            "parity_rel_l2_sampled": par, "tolerance": {"f32": 1e-5, "f32_cuda": 1e-5, "f16": 5e-3, "bf16": 5e-3, "f32_frec": 1e-5,
                          "f16_frec": 5e-3},
            "variants": variants, "rows": rows, "input_generation_s": t_gen,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

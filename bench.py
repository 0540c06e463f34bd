#!/usr/bin/env python
"""Benchmark: even-odd CG solve of the twisted-mass Wilson matrix to a 1e-10
true residual on a 24^3 x 48 lattice (near-identity links exp(i eps H),
eps = 0.3, kappa = 0.16, 2 kappa mu = 0.005, Gaussian source).

One step is one complete solve through the library (source preparation, CG
iterations of half hops + BLAS-1 with fused reductions, reconstruction, FP64
true residual).  Prints ONE JSON line (rank 0):

  value    whole-job algorithmic GB/s of the solve (library work counters:
           every kernel's inputs read once, outputs written once) over the
           device-timed region, summed over ranks / max time over ranks
  roofline the half-hop kernel timed alone with CUDA events on the library
           stream; FP64 arithmetic is bound by the FP64 pipe (bound "alu":
           peak derived from this device's SM count and maximum clock, and
           peak_measured from the library's FMA microbenchmark),
           float-float and lower precisions by HBM
  hmc      time per HMC trajectory, dH and acceptance: Nf=2 leapfrog on
           16^3 x 32, and the paper's setup C (tlSym, 2MN) on 24^3 x 8
  config3  the 32^3 x 64 heatbath workload: time to 1e-10 for FP64 and the
           mixed paths (FP64 and float-float outer), and its 12 point
           sources as one 12-RHS solve against 12 single solves
  cg       the FP64 solve's iterations and true residual, and
           cg.variants: time to 1e-10 for every precision path on the same
           system (FP64, FP64 outer / FP32 inner, float-float, float-float
           outer with FP32 / FP16+scale / BF16+scale inner), and
           cg.multi_rhs: the 12 point sources in one 12-RHS solve against 12
           single-RHS solves
  e2e      the same metric through the public API with host buffers: links
           and source copied host->device, gauge import, solve, solution
           copied device->host, all inside the timed region
  cpu_baseline  the FP64 oracle (C + OpenMP) running a bounded number of CG
           iterations of the same system on the host cores

--impl reference times the oracle itself on the same workload (the paper has
no runnable reference implementation).  --gpus N > 1 runs N independent
replicas (the library solves each system on one GPU; there is no sharded solve).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s (% HBM peak); CG time-to-1e-10 residual, FP64 vs mixed/multi-RHS"
WORKLOAD = {"workload": "24^3x48 twisted-mass Wilson even-odd CG to 1e-10 true residual",
            "lattice": [24, 24, 24, 48], "links": "exp(i eps H), eps=0.3", "kappa": 0.16,
            "two_kappa_mu": 0.005, "source": "Gaussian", "bc": "antiperiodic t"}
L = (24, 24, 24, 48)
KAPPA = 0.16
MU = 0.005 / (2 * 0.16)
TOL = 1e-10
SEED_U, SEED_B = 2001, 2002
FP64_FMA_PER_CLK_PER_SM = 2  # GB300's FP64 pipe: 2 FP64 FMA per clock per SM
PREC_NAMES = {"f64": 0, "df64": 1, "f32": 2, "bf16s": 3, "f16s": 4}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def reduce_over_ranks(dist, t_local, bytes_local, device):
    """Whole-job figures of N independent replicas: the slowest rank's time
    (max) and the bytes of all ranks (sum).  dist = None for one process."""
    if dist is None:
        return t_local, bytes_local
    import torch
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    bb = torch.tensor([bytes_local], device=device, dtype=torch.float64)
    dist.all_reduce(bb, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(bb.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs():
    from paper_1209_5942_gb300 import inputs
    U = inputs.random_gauge(L, "near", seed=SEED_U, eps=0.3)
    b = inputs.gaussian_spinor(L, SEED_B)
    return U, b


# ------------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle on the host cores
# ------------------------------------------------------------------------------

def bytes_per_cg_iteration(Vh: int) -> float:
    """Algorithmic bytes of one CG iteration in FP64 (2 Mhat + 2 Mhat^+ = 4 half
    hops, two of them with the fused A psi term; x/s update; p update)."""
    hop = 8 * 144 + 192 + 192
    return Vh * (2 * hop + 2 * (hop + 192) + 6 * 192 + 3 * 192)


def oracle_sample(U, b, iters: int):
    from oracle import oracle
    t0 = time.perf_counter()
    bhat = oracle.eo_prepare(U, b, L, KAPPA, MU)
    t1 = time.perf_counter()
    oracle.cg_fixed_iters(U, bhat, L, KAPPA, MU, iters)
    t2 = time.perf_counter()
    return t2 - t1, t1 - t0


def cpu_cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    from oracle import oracle
    oracle.build()
    U, b = make_inputs()
    Vh = int(np.prod(L)) // 2
    iters = args.ref_iters
    for _ in range(args.warmup):
        oracle_sample(U, b, 1)
    times = []
    for _ in range(args.steps):
        t, _ = oracle_sample(U, b, iters)
        times.append(t)
    tot = sum(times)
    gbs = bytes_per_cg_iteration(Vh) * iters * len(times) / tot / 1e9
    sample = f"{iters} CG iterations (2 Mhat + 2 Mhat^+ each) of the 24^3x48 system per step"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------

def run_gpu(args):
    import torch

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1209_5942_gb300 import build, lqcd
    build.build()
    ctx = lqcd.Context(local)
    stream = torch.cuda.current_stream(local)
    prec = PREC_NAMES[args.prec]
    inner = PREC_NAMES[args.inner] if args.inner else prec
    recon = args.recon

    U_h, b_h = make_inputs()
    V = int(np.prod(L))
    Vh = V // 2
    U_d = torch.from_numpy(U_h).cuda()
    # a mixed solve keeps 18-real links for its FP64-class operator (ALU-bound
    # on GB300, so rebuilding rows costs time) and uses `recon` for the sloppy one
    G = lqcd.lqcd_gauge_import(ctx, U_d, L, recon=recon if inner == prec else 18)
    # the field in the sloppy operator's link format, for timing that operator's hop
    Gh = G if (inner == prec or recon == 18) else lqcd.lqcd_gauge_import(ctx, U_d, L, recon=recon)
    del U_d
    b_d = torch.from_numpy(b_h).cuda()
    bd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    xd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    fb = lqcd.field(bd, lqcd.LQCD_LAYOUT_EO)
    fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO)
    lqcd.lqcd_spinor_pack(ctx, L, b_d, fb)
    prm = lqcd.cg_params(tol=TOL, outer_prec=prec, inner_prec=inner, max_iter=50000,
                         check_every=args.check_every, sloppy_recon=recon)

    def step():
        return lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm)

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nvtx_push("timed_solves")  # ncu --nvtx --nvtx-include timed_solves/ captures the timed steps
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step()[0])
    e1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    t, bytes_total = reduce_over_ranks(dist, ms / 1e3, cnt.bytes, "cuda")
    value = bytes_total / t / 1e9

    # dominant kernel: the half hop of the solve, timed alone on the library stream
    hop = time_half_hop(ctx, Gh, lqcd, torch, inner, recon, stream)

    # end to end through the public API with host buffers
    e2e = run_e2e(ctx, lqcd, torch, U_h, b_h, prm, recon, args, stream)

    peaks, peak_kind = measured_peaks()
    if args.traffic is None:
        args.traffic = NCU_TRAFFIC.get((hop["kernel"], tuple(L), inner, recon))
    # FP64 pipe peak derived from this device's SM count and maximum SM clock,
    # and the FMA rate measured by the library's microbenchmark on this GPU
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    fp64_derived = sms * FP64_FMA_PER_CLK_PER_SM * 2 * max_mhz * 1e6 / 1e12
    fp64_meas, fp32_meas = lqcd.lqcd_measure_peaks(ctx)
    if inner == lqcd.LQCD_F64:
        roof = {"bound": "alu", "achieved": hop["tflops"], "peak": fp64_derived, "unit": "TFLOP/s",
                "frac": hop["tflops"] / fp64_derived, "traffic": args.traffic,
                "peak_kind": f"derived: {sms} SMs x {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk x 2 x "
                             f"{max_mhz:.0f} MHz",
                "peak_measured": fp64_meas, "frac_of_measured": hop["tflops"] / fp64_meas,
                "peak_measured_kind": "lqcd_measure_peaks: FP64 FMA chains, 8 x 256 threads per SM",
                "hbm_GBs": hop["gbs"], "hbm_frac": hop["gbs"] / peaks["hbm_gbs"]}
    else:
        roof = {"bound": "hbm", "achieved": hop["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hop["gbs"] / peaks["hbm_gbs"], "traffic": args.traffic,
                "peak_kind": f"{peak_kind} (copy bandwidth, burst)", "tflops": hop["tflops"]}
    roof["kernel"] = hop["kernel"]
    roof["bytes_per_launch"] = hop["bytes"]
    roof["ms_per_launch"] = hop["ms"]

    roof["fp32_peak_measured_TFLOPs"] = fp32_meas
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "df64 (float-float)", 2: "f32", 3: "bf16+scale", 4: "f16+scale"}[inner]
            + ("" if inner == prec else f" inner / {args.prec} outer"),
            "data": "synthetic",
            "config": dict(WORKLOAD, outer_prec=args.prec, inner_prec=args.inner or args.prec,
                           recon=recon, l2="inputs larger than L2 (links 382 MB)",
                           parallelism=f"replicas x{world}"),
            "cg": {"iters": stats[-1]["iters"], "true_resid": stats[-1]["true_resid"],
                   "reliable_updates": stats[-1]["reliable_updates"],
                   "time_to_solution_s": ms / 1e3 / args.steps,
                   "pct_hbm_solve": 100.0 * value / world / peaks["hbm_gbs"]},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(cnt.launches),
            "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(U_h, b_h, args)
    if rank == 0 and not args.no_variants:
        t_f64 = ms / 1e3 / args.steps
        line["cg"]["variants"] = run_variants(ctx, G, fb, fx, lqcd, torch, t_f64, args.variants)
        line["cg"]["multi_rhs"] = run_multi_rhs(ctx, G, lqcd, torch)
        del G, Gh
        line["config3"] = run_config3_block(ctx, lqcd, torch, args.sweeps)
        line["hmc"] = run_hmc_block(ctx, lqcd, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def ctypes_byref(x):
    import ctypes
    return ctypes.byref(x)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# half hop timed by time_half_hop, from one ncu capture of that launch (the
# FP64 half hop on 24^3 x 48 with 18-real links); valid only for the kernel as
# captured.
NCU_TRAFFIC = {("hop_kernel prec=0 recon=18", (24, 24, 24, 48), 0, 18): 503709952.0}


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def time_half_hop(ctx, G, lqcd, torch, prec, recon, stream, reps=30):
    """Average duration of the half hop (no epilogue) with CUDA events."""
    n_half, sb = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
    gen = torch.Generator(device="cuda").manual_seed(7)
    if sb:  # 16-bit values in [-1, 1) with unit site scales
        din = torch.zeros(n_half // 8, dtype=torch.float64, device="cuda")
    else:   # Gaussian reals (F64 / F32; DF64 high and low words alike)
        din = torch.randn(n_half // 8, dtype=torch.float64, device="cuda", generator=gen)
        if prec != lqcd.LQCD_F64:
            din = torch.randn(n_half // 4, dtype=torch.float32, device="cuda", generator=gen).view(torch.float64)
    dout = torch.zeros_like(din)
    s_in = torch.ones(max(sb // 4, 1), dtype=torch.float32, device="cuda") if sb else None
    s_out = torch.zeros_like(s_in) if sb else None
    fi = lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec, 1, s_in)
    fo = lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec, 1, s_out)
    for _ in range(5):
        lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
    torch.cuda.synchronize()
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nvtx_push("half_hop")  # ncu --nvtx --nvtx-include half_hop/ captures these launches
    e0.record(stream)
    for _ in range(reps):
        lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
    e1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    bytes_per = cnt.hop_bytes / reps
    flops_per = cnt.hop_flops / reps
    return {"kernel": f"hop_kernel prec={prec} recon={recon}", "ms": ms, "bytes": bytes_per,
            "gbs": bytes_per / (ms / 1e3) / 1e9, "tflops": flops_per / (ms / 1e3) / 1e12}


def run_e2e(ctx, lqcd, torch, U_h, b_h, prm, recon, args, stream):
    """Public-API step with host buffers: H2D of links and source, import, solve, D2H."""
    import_recon = recon if prm.inner_prec == prm.outer_prec else 18
    U_pin = torch.from_numpy(U_h).pin_memory()
    b_pin = torch.from_numpy(b_h).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    U_dev = torch.empty(U_pin.shape, dtype=U_pin.dtype, device="cuda")
    b_dev = torch.empty(b_pin.shape, dtype=b_pin.dtype, device="cuda")
    x_dev = torch.empty_like(b_dev)

    def step():
        U_dev.copy_(U_pin, non_blocking=True)
        b_dev.copy_(b_pin, non_blocking=True)
        G = lqcd.lqcd_gauge_import(ctx, U_dev, L, recon=import_recon)
        lqcd.lqcd_cg_solve(ctx, G, lqcd.field(b_dev, lqcd.LQCD_LAYOUT_LEXI),
                           lqcd.field(x_dev, lqcd.LQCD_LAYOUT_LEXI), KAPPA, MU, prm)
        x_pin.copy_(x_dev, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        G.free()

    step()
    n = max(1, min(args.steps, 3))
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    bi = U_pin.numel() * 16 + b_pin.numel() * 16
    bo = x_pin.numel() * 16
    return {"value": cnt.bytes / wall / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(bi),
            "d2h_bytes_per_step": int(bo), "ms_per_step": 1e3 * wall / n, "steps": n,
            "note": "algorithmic bytes of the library kernels / wall time including copies and import"}


def cpu_baseline(U_h, b_h, args):
    from oracle import oracle
    oracle.build()
    Vh = int(np.prod(L)) // 2
    iters = args.ref_iters
    t, tprep = oracle_sample(U_h, b_h, iters)
    return {"value": bytes_per_cg_iteration(Vh) * iters / t / 1e9, "unit": "GB/s",
            "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{iters} CG iterations (2 Mhat + 2 Mhat^+ each) of the 24^3x48 system, "
                      f"{t:.1f} s; GB/s counted with the same algorithmic bytes per iteration"}


def _timed_solve(ctx, G, fb, fx, lqcd, torch, prm):
    """One warm-up solve (autotuning, graph capture) and one solve timed with
    CUDA events on the library stream; returns (seconds, stats)."""
    lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm, allow_noconv=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    st = lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm, allow_noconv=True)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, st


def run_variants(ctx, G, fb, fx, lqcd, torch, t_f64, with_bicgstab=False):
    """Time to a 1e-10 true residual on the same 24^3 x 48 system for every
    precision path: plain IEEE FP64, mixed with IEEE-FP64 reliable updates,
    float-float, and float-float outer with FP32 / FP16+scale / BF16+scale
    inner solves (inner operator on REC12 links).  Each entry carries the
    library's recomputed IEEE-FP64 true residual."""
    out = {}
    combos = [("f64", "f64", 18), ("f64", "f32", 12), ("df64", "df64", 18), ("df64", "f32", 12),
              ("df64", "f16s", 12), ("df64", "bf16s", 12)]
    if with_bicgstab:
        combos += [("f64", "f64", 18, "bicgstab"), ("df64", "df64", 18, "bicgstab"),
                   ("df64", "f32", 12, "bicgstab")]
    for combo in combos:
        outer, inner, recon = combo[:3]
        bicg = len(combo) > 3
        prm = lqcd.cg_params(tol=TOL, outer_prec=PREC_NAMES[outer], inner_prec=PREC_NAMES[inner],
                             max_iter=50000 if not bicg else 4000, max_restarts=10, sloppy_recon=recon,
                             check_every=20,
                             solver=lqcd.LQCD_SOLVER_BICGSTAB if bicg else lqcd.LQCD_SOLVER_CG)
        key = f"{outer}/{inner}" + ("/bicgstab" if bicg else "")
        try:
            t, st = _timed_solve(ctx, G, fb, fx, lqcd, torch, prm)
            st = st[0]
            out[key] = {"time_to_solution_s": t, "iters": st["iters"],
                        "reliable_updates": st["reliable_updates"], "restarts": st["restarts"],
                        "converged": st["converged"], "true_resid": st["true_resid"],
                        "speedup_vs_f64_cg": t_f64 / t}
        except Exception as e:  # report, do not hide
            out[key] = {"error": str(e)}
    return out


def run_multi_rhs(ctx, G, lqcd, torch, nrhs=12):
    """The 12 unit point sources (spin x colour at the origin) on the same
    24^3 x 48 field: one 12-RHS solve against 12 single-RHS solves, in
    float-float / FP32 and float-float / BF16 mixed precision and in
    float-float."""
    from paper_1209_5942_gb300 import inputs
    b12 = inputs.point_sources(L)
    out = {}
    for outer, inner, recon in (("df64", "f32", 12), ("df64", "bf16s", 12), ("df64", "df64", 18)):
        prm = lqcd.cg_params(tol=TOL, outer_prec=PREC_NAMES[outer], inner_prec=PREC_NAMES[inner],
                             max_iter=50000, sloppy_recon=recon, check_every=20)
        bd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, nrhs)
        xd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, nrhs)
        fb = lqcd.field(bd, lqcd.LQCD_LAYOUT_EO, nrhs=nrhs)
        fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO, nrhs=nrhs)
        lqcd.lqcd_spinor_pack(ctx, L, torch.from_numpy(b12).cuda(), fb)
        t_multi, st = _timed_solve(ctx, G, fb, fx, lqcd, torch, prm)
        b1, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        x1, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        f1 = lqcd.field(b1, lqcd.LQCD_LAYOUT_EO)
        g1 = lqcd.field(x1, lqcd.LQCD_LAYOUT_EO)
        t_seq, st_seq = 0.0, []
        for r in range(nrhs):
            lqcd.lqcd_spinor_pack(ctx, L, torch.from_numpy(b12[r]).cuda(), f1)
            t, s1 = _timed_solve(ctx, G, f1, g1, lqcd, torch, prm)
            t_seq += t
            st_seq.append(s1[0])
        out[f"{outer}/{inner}"] = {
            "nrhs": nrhs, "multi_rhs_s": t_multi, "sequential_s": t_seq, "speedup": t_seq / t_multi,
            "iters_max": max(s["iters"] for s in st), "iters_max_sequential": max(s["iters"] for s in st_seq),
            "true_resid_max": max(s["true_resid"] for s in st),
            "converged": all(s["converged"] for s in st)}
        del bd, xd, b1, x1
    return out


def run_config3_block(ctx, lqcd, torch, sweeps):
    """The mixed-precision workload on 32^3 x 64 (heatbath field at beta = 5.7
    from a cold start, kappa = 0.157, 2 kappa mu = 0.003, Gaussian source):
    time to a 1e-10 true residual for plain FP64 and for FP32 / BF16+scale /
    FP16+scale inner solves with IEEE-FP64 reliable updates, the same with a
    float-float outer, and on the same field the 12 unit point sources in one
    12-RHS mixed solve against 12 single-RHS solves."""
    from paper_1209_5942_gb300 import inputs
    Lc = (32, 32, 32, 64)
    kappa, mu = 0.157, 0.003 / (2 * 0.157)
    G, thb, plaq = _heatbath_field(torch, lqcd, ctx, Lc, 5.7, sweeps, 3003)
    b = inputs.gaussian_spinor(Lc, 3004)
    sol = _solve_variants(torch, lqcd, ctx, G, Lc, b, kappa, mu,
                          [("f64", "f64", 18), ("f64", "f32", 12), ("f64", "bf16s", 12), ("f64", "f16s", 12),
                           ("df64", "df64", 18), ("df64", "f32", 12), ("df64", "bf16s", 12),
                           ("df64", "f16s", 12)])
    t64 = sol["f64/f64/rec18"].get("time_to_solution_s")
    for v in sol.values():
        if t64 and v.get("time_to_solution_s"):
            v["speedup_vs_f64_cg"] = t64 / v["time_to_solution_s"]
        v.pop("solve_GBs", None)
    b12 = inputs.point_sources(Lc)
    multi = _solve_variants(torch, lqcd, ctx, G, Lc, b12, kappa, mu, [("df64", "f32", 12)], nrhs=12)
    seq_t, seq_it = 0.0, 0
    for r in range(12):
        v = list(_solve_variants(torch, lqcd, ctx, G, Lc, b12[r], kappa, mu, [("df64", "f32", 12)]).values())[0]
        seq_t += v["time_to_solution_s"]
        seq_it = max(seq_it, v["iters"])
    m = multi["df64/f32/rec12"]
    G.free()
    return {"workload": f"32^3x64, {sweeps} CM heatbath sweeps beta=5.7 from cold (plaquette {plaq:.4f}), "
                        "kappa=0.157, 2 kappa mu=0.003, Gaussian source, 1e-10 true residual",
            "heatbath_s": thb, "solves": sol,
            "multi_rhs_12_point_sources": {"multi_rhs_s": m["time_to_solution_s"], "sequential_s": seq_t,
                                           "speedup": seq_t / m["time_to_solution_s"], "iters_max": m["iters"],
                                           "iters_max_sequential": seq_it,
                                           "true_resid_max": m["true_resid_max"],
                                           "converged": m["converged"]}}


def _trajectories(torch, lqcd, ctx, G, make_params, n_therm, n_meas):
    out = []
    for t in range(n_therm + n_meas):
        st = lqcd.lqcd_hmc_trajectory(ctx, G, make_params(t))
        if t >= n_therm:
            out.append(st)
    return {"s_per_trajectory": statistics.median(s["seconds"] for s in out),
            "dH": [s["dH"] for s in out], "accepted": [s["accepted"] for s in out],
            "cg_iters_per_trajectory": [s["cg_iters"] for s in out],
            "plaquette": [s["plaquette"] for s in out], "thermalisation_trajectories": n_therm}


def run_hmc_block(ctx, lqcd, torch):
    """Two HMC workloads (time per trajectory with every force through the
    library's solver and adjoint kernels; H and dH in FP64): the Nf = 2
    twisted-mass leapfrog run on 16^3 x 32 (beta 5.6, kappa 0.16, 2 kappa mu
    0.005, tau 1, 20 steps) and the paper's setup C on 24^3 x 8 (tlSym
    beta 3.9, kappa 0.160856, a mu 0.1, 2MN 10 fermion x 10 gauge steps,
    float-float gauge force and link update), each started from the
    library's heatbath and thermalised with a few trajectories."""
    cg = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32, sloppy_recon=18,
                        check_every=20)
    out = {}
    L5 = (16, 16, 16, 32)
    G, _, _ = _heatbath_field(torch, lqcd, ctx, L5, 5.6, 50, 5005)
    out["nf2_leapfrog_16x32"] = _trajectories(
        torch, lqcd, ctx, G,
        lambda t: lqcd.hmc_params(5.6, 0.16, 0.005 / 0.32, tau=1.0, nsteps=20, nf=1, seed=6006, traj=t, cg=cg),
        2, 3)
    out["nf2_leapfrog_16x32"]["workload"] = ("16^3x32, Wilson beta=5.6, kappa=0.16, 2 kappa mu=0.005, leapfrog "
                                            "tau=1 20 steps, 50 heatbath sweeps from cold, DF64/F32 CG to 1e-10")
    G.free()
    LC = (24, 24, 24, 8)
    G, _, _ = _heatbath_field(torch, lqcd, ctx, LC, 6.0, 100, 5105)
    out["setup_C_24x8"] = _trajectories(
        torch, lqcd, ctx, G,
        lambda t: lqcd.hmc_params(3.9, 0.160856, 0.1, tau=1.0, nsteps=10, nf=1, seed=6106, traj=t, cg=cg,
                                  integrator=lqcd.LQCD_2MN, c1=lqcd.TLSYM_C1, nsteps_gauge=10,
                                  force_prec=lqcd.LQCD_DF64),
        2, 4)
    out["setup_C_24x8"]["workload"] = ("24^3x8, tlSym beta=3.9, kappa=0.160856, a mu=0.1, 2MN 10 fermion x 10 gauge "
                                      "steps, tau=1, float-float gauge force and link update, DF64/F32 CG to "
                                      "1e-10; 100 Wilson heatbath sweeps at beta=6.0 from cold")
    G.free()
    return out


# ------------------------------------------------------------------------------
# The other workloads (--config): one JSON line each, same keys where they apply
# ------------------------------------------------------------------------------

def _gpu_setup():
    import torch
    from paper_1209_5942_gb300 import build, lqcd
    build.build()
    torch.cuda.set_device(0)
    return torch, lqcd, lqcd.Context(0)


def _timed(torch, fn, reps=1):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps, out


def _heatbath_field(torch, lqcd, ctx, L, beta, sweeps, seed):
    """Cold start + `sweeps` Cabibbo-Marinari sweeps with the library's heatbath."""
    from paper_1209_5942_gb300 import inputs
    G = lqcd.lqcd_gauge_import(ctx, torch.from_numpy(inputs.random_gauge(L, "cold")).cuda(), L,
                               recon=18)
    t, _ = _timed(torch, lambda: [lqcd.lqcd_heatbath_sweep(ctx, G, beta, seed, s)
                                  for s in range(sweeps)])
    return G, t, lqcd.lqcd_plaquette(ctx, G)


def _solve_variants(torch, lqcd, ctx, G, L, b_h, kappa, mu, combos, nrhs=1, reps=1):
    bd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, nrhs)
    xd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, nrhs)
    fb = lqcd.field(bd, lqcd.LQCD_LAYOUT_EO, nrhs=nrhs)
    fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO, nrhs=nrhs)
    lqcd.lqcd_spinor_pack(ctx, L, torch.from_numpy(b_h).cuda(), fb)
    out = {}
    for combo in combos:
        outer, inner, recon = combo[:3]
        solver = combo[3] if len(combo) > 3 else "cg"
        prm = lqcd.cg_params(tol=TOL, outer_prec=PREC_NAMES[outer], inner_prec=PREC_NAMES[inner],
                             max_iter=100000, sloppy_recon=recon, check_every=20, max_restarts=10,
                             solver=lqcd.LQCD_SOLVER_BICGSTAB if solver == "bicgstab" else lqcd.LQCD_SOLVER_CG)
        name = f"{outer}/{inner}/rec{recon}" + ("/bicgstab" if solver == "bicgstab" else "")
        try:
            # warm-up (autotuning, graph); non-convergence is reported, not hidden
            lqcd.lqcd_cg_solve(ctx, G, fb, fx, kappa, mu, prm, allow_noconv=True)
            lqcd.lib().lqcd_reset_counters(ctx.handle)
            # NVTX range for profiling, e.g. ncu --nvtx --nvtx-include "solve_12rhs_df64_f32_rec12/"
            nvtx_push(f"solve_{nrhs}rhs_" + name.replace("/", "_"))
            t, st = _timed(torch, lambda: lqcd.lqcd_cg_solve(ctx, G, fb, fx, kappa, mu, prm,
                                                             allow_noconv=True), reps)
            nvtx_pop()
        except Exception as e:
            out[name] = {"error": str(e)}
            continue
        cnt = lqcd.lqcd_counters()
        lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
        out[name] = {
            "time_to_solution_s": t, "iters": max(s["iters"] for s in st),
            "reliable_updates": st[0]["reliable_updates"], "restarts": st[0]["restarts"],
            "converged": all(s["converged"] for s in st),
            "true_resid_max": max(s["true_resid"] for s in st),
            "solve_GBs": cnt.bytes / reps / t / 1e9}
    return out


def config_line(name, metric_value, extra, workload):
    line = {"metric": METRIC, "value": metric_value, "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "config": workload}
    line.update(extra)
    line["config_name"] = name
    print(json.dumps(line), flush=True)


def run_config(args):
    torch, lqcd, ctx = _gpu_setup()
    from paper_1209_5942_gb300 import inputs
    peaks, _ = measured_peaks()
    c = args.config
    if c == "1":
        Lc = (4, 4, 4, 4)
        kappa, mu = 0.15, 0.01 / 0.3
        U = inputs.random_gauge(Lc, "haar", seed=1001)
        G = lqcd.lqcd_gauge_import(ctx, torch.from_numpy(U).cuda(), Lc)
        b = inputs.gaussian_spinor(Lc, 1002)
        bd = torch.from_numpy(b).cuda()
        out = torch.zeros_like(bd)
        fi = lqcd.field(bd, lqcd.LQCD_LAYOUT_LEXI)
        fo = lqcd.field(out, lqcd.LQCD_LAYOUT_LEXI)
        lqcd.lqcd_apply_M(ctx, G, fi, fo, kappa, mu)
        t_m, _ = _timed(torch, lambda: lqcd.lqcd_apply_M(ctx, G, fi, fo, kappa, mu), 200)
        sol = _solve_variants(torch, lqcd, ctx, G, Lc, b, kappa, mu, [("f64", "f64", 18)], reps=5)
        config_line("4^4 latency", None, {"apply_M_lexi_us": 1e6 * t_m, "solve": sol},
                    {"workload": "4^4 Haar, kappa=0.15, 2 kappa mu=0.01 (launch-latency bound)"})
    elif c == "3":
        Lc = (32, 32, 32, 64)
        kappa, mu = 0.157, 0.003 / (2 * 0.157)
        G, thb, plaq = _heatbath_field(torch, lqcd, ctx, Lc, 5.7, args.sweeps, 3003)
        b = inputs.gaussian_spinor(Lc, 3004)
        sol = _solve_variants(torch, lqcd, ctx, G, Lc, b, kappa, mu,
                              [("f64", "f64", 18), ("df64", "df64", 18), ("df64", "f32", 12),
                               ("df64", "bf16s", 12), ("df64", "f16s", 12),
                               ("f64", "f64", 18, "bicgstab"), ("df64", "df64", 18, "bicgstab"),
                               ("df64", "f32", 12, "bicgstab"), ("df64", "f16s", 12, "bicgstab")])
        ok = [v for v in sol.values() if v.get("converged")]
        best = min(v["time_to_solution_s"] for v in ok) if ok else None
        config_line("32^3x64 mixed precision", sol["df64/f32/rec12"].get("solve_GBs"),
                    {"heatbath_s": thb, "heatbath_sweeps": args.sweeps, "plaquette": plaq,
                     "solves": sol, "fastest_time_to_solution_s": best},
                    {"workload": f"32^3x64, {args.sweeps} CM heatbath sweeps beta=5.7 cold start, "
                                 "kappa=0.157, 2 kappa mu=0.003, Gaussian source, 1e-10"})
    elif c == "4a":
        Lc = (32, 32, 32, 64)
        kappa, mu = 0.157, 0.003 / (2 * 0.157)
        G, thb, plaq = _heatbath_field(torch, lqcd, ctx, Lc, 5.7, args.sweeps, 3003)
        b12 = inputs.point_sources(Lc)
        multi = _solve_variants(torch, lqcd, ctx, G, Lc, b12, kappa, mu,
                                [("df64", "f32", 12), ("df64", "df64", 18)], nrhs=12)
        seq = {}
        for outer, inner, recon in [("df64", "f32", 12), ("f64", "f64", 18)]:
            ts, its = 0.0, 0
            for r in range(12 if not args.quick else 2):
                s1 = _solve_variants(torch, lqcd, ctx, G, Lc, b12[r], kappa, mu, [(outer, inner, recon)])
                v = list(s1.values())[0]
                ts += v["time_to_solution_s"]
                its = max(its, v["iters"])
            if args.quick:
                ts *= 6
            seq[f"{outer}/{inner}/rec{recon} x12 sequential"] = {"time_s": ts, "iters_max": its}
        hop = time_hop_multi(ctx, G, lqcd, torch, Lc, 12)
        config_line("12 point sources, multi-RHS", hop["gbs"],
                    {"multi_rhs": multi, "sequential": seq, "hop_multi_rhs": hop, "plaquette": plaq},
                    {"workload": "32^3x64 heatbath field (beta=5.7), 12 unit point sources, "
                                 "kappa=0.157, 2 kappa mu=0.003, 1e-10"})
    elif c == "4b":
        shapes = [(8, 8, 8, 8)] * 8 + [(12, 12, 12, 24)] * 8 + [(16, 16, 16, 32)] * 8 + [(20, 20, 20, 40)] * 8
        kappa, mu = 0.16, 0.005 / 0.32
        Gs, fbs, fxs, keep = [], [], [], []
        for k, Lk in enumerate(shapes):
            U = inputs.random_gauge(Lk, "near", seed=4000 + k, eps=0.3)
            G = lqcd.lqcd_gauge_import(ctx, torch.from_numpy(U).cuda(), Lk, recon=18)
            bd, _ = lqcd.alloc_field(Lk, lqcd.LQCD_FULL, lqcd.LQCD_F64)
            xd, _ = lqcd.alloc_field(Lk, lqcd.LQCD_FULL, lqcd.LQCD_F64)
            fb = lqcd.field(bd, lqcd.LQCD_LAYOUT_EO)
            lqcd.lqcd_spinor_pack(ctx, Lk, torch.from_numpy(inputs.gaussian_spinor(Lk, 5000 + k)).cuda(), fb)
            Gs.append(G)
            fbs.append(fb)
            fxs.append(lqcd.field(xd, lqcd.LQCD_LAYOUT_EO))
        prm = lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32,
                             sloppy_recon=12, check_every=20)
        n = len(shapes)
        batch = lambda: lqcd.lqcd_cg_solve_batch(ctx, Gs, fbs, fxs, [kappa] * n, [mu] * n, prm)
        batch()
        lqcd.lib().lqcd_reset_counters(ctx.handle)
        tb, st = _timed(torch, batch)
        cnt = lqcd.lqcd_counters()
        lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
        loop = lambda: [lqcd.lqcd_cg_solve(ctx, Gs[k], fbs[k], fxs[k], kappa, mu, prm) for k in range(n)]
        loop()
        tl, _ = _timed(torch, loop)
        config_line("uneven batch", cnt.bytes / tb / 1e9,
                    {"batched_s": tb, "loop_s": tl, "speedup": tl / tb,
                     "iters_max": max(s["iters"] for s in st),
                     "true_resid_max": max(s["true_resid"] for s in st), "gpu_launches": int(cnt.launches)},
                    {"workload": "8 each of 8^4, 12^3x24, 16^3x32, 20^3x40 (sum V = 3973120), "
                                 "exp(i 0.3 H) links, kappa=0.16, 2 kappa mu=0.005, F32 inner / DF64 outer"})
    elif c == "5":
        Lc = (16, 16, 16, 32)
        beta, kappa, mu = 5.6, 0.16, 0.005 / 0.32
        G, thb, plaq0 = _heatbath_field(torch, lqcd, ctx, Lc, beta, args.sweeps, 5005)
        cg = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32,
                            sloppy_recon=18, check_every=20)
        trajs, therm = [], []
        for t in range(args.therm + args.trajs):
            st = lqcd.lqcd_hmc_trajectory(ctx, G, lqcd.hmc_params(beta, kappa, mu, tau=1.0, nsteps=20,
                                                                   nf=1, seed=6006, traj=t, cg=cg))
            (therm if t < args.therm else trajs).append(st)
        secs = [s["seconds"] for s in trajs[1:]] or [trajs[0]["seconds"]]
        # the same ensemble continued with 2MN on three time scales and mass
        # preconditioning (mu2 = 10 mu): ratio force 5 steps, W force 2, gauge 2
        imp = []
        for t in range(args.trajs):
            imp.append(lqcd.lqcd_hmc_trajectory(ctx, G, lqcd.hmc_params(
                beta, kappa, mu, tau=1.0, nsteps=5, nf=1, seed=6007, traj=t, cg=cg,
                integrator=lqcd.LQCD_2MN, nsteps_gauge=2, mu2=10 * mu, nsteps_mid=2)))
        isecs = [s["seconds"] for s in imp[1:]] or [imp[0]["seconds"]]
        improved = {"integrator": "2MN ratio/W/gauge = 5/2/2 steps, mu2 = 10 mu",
                    "s_per_trajectory": statistics.median(isecs), "dH": [s["dH"] for s in imp],
                    "acceptance": sum(s["accepted"] for s in imp) / len(imp),
                    "cg_iters_per_trajectory": [s["cg_iters"] for s in imp],
                    "plaquette": [s["plaquette"] for s in imp]}
        config_line("Nf=2 HMC", None,
                    {"s_per_trajectory": statistics.median(secs),
                     "dH": [s["dH"] for s in trajs], "accepted": [s["accepted"] for s in trajs],
                     "acceptance": sum(s["accepted"] for s in trajs) / len(trajs),
                     "cg_iters_per_trajectory": [s["cg_iters"] for s in trajs],
                     "exp_minus_dH_mean": float(np.mean([np.exp(-s["dH"]) for s in trajs])),
                     "plaquette": [s["plaquette"] for s in trajs], "plaquette_after_heatbath": plaq0,
                     "heatbath_s": thb, "thermalisation_trajectories": len(therm),
                     "thermalisation_dH": [s["dH"] for s in therm],
                     "thermalisation_plaquette": [s["plaquette"] for s in therm],
                     "mass_preconditioned_2mn": improved},
                    {"workload": f"16^3x32, beta=5.6, kappa=0.16, 2 kappa mu=0.005, {args.sweeps} "
                                 "heatbath sweeps from cold, leapfrog tau=1 20 steps, "
                                 "F32-inner/DF64 CG to 1e-10 per force"})
    elif c == "C":
        # the paper's HMC setup C (Table "setup", Sec. 5.3): tlSym action, beta = 3.9,
        # kappa = kappa_c = 0.160856, a mu = 0.1, 2MN with 10 steps on the fermion and
        # on the gauge time scale, tau = 1, on 24^3 x 8; started from our own
        # configuration (Wilson heatbath at beta = 6.0, whose plaquette is near the
        # tlSym beta = 3.9 value) and thermalised with HMC before measuring
        Lc = (24, 24, 24, 8)
        beta, kappa, mu, c1 = 3.9, 0.160856, 0.1, lqcd.TLSYM_C1
        G, thb, plaq0 = _heatbath_field(torch, lqcd, ctx, Lc, 6.0, min(args.sweeps, 100), 5105)
        cg = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32,
                            sloppy_recon=18, check_every=20)
        trajs, therm = [], []
        for t in range(args.therm + args.trajs):
            st = lqcd.lqcd_hmc_trajectory(ctx, G, lqcd.hmc_params(
                beta, kappa, mu, tau=1.0, nsteps=10, nf=1, seed=6106, traj=t, cg=cg,
                integrator=lqcd.LQCD_2MN, c1=c1, nsteps_gauge=10, force_prec=PREC_NAMES[args.force_prec]))
            (therm if t < args.therm else trajs).append(st)
        secs = [s["seconds"] for s in trajs[1:]] or [trajs[0]["seconds"]]
        F = torch.zeros((4, int(np.prod(Lc)), 8), dtype=torch.float64, device="cuda")
        gf = {}
        for name, cc in (("tlsym", c1), ("wilson", 0.0)):
            for pn in ("f64", "df64"):
                gf[f"{name}_{pn}"] = 1e3 * _timed(torch, lambda: lqcd.lqcd_gauge_force(
                    ctx, G, beta, F, want_action=False, c1=cc, prec=PREC_NAMES[pn]), 5)[0]
        # the fermion force with a cached solution X: the adjoint kernel plus the
        # operators that build Y = Mhat X, W_o and Z_o (no CG); the paper counts
        # 4736 B and 1748 flop per site and direction for its force kernel
        Vc = int(np.prod(Lc))
        full_d, _ = lqcd.alloc_field(Lc, lqcd.LQCD_FULL, lqcd.LQCD_F64)  # Gaussian on the even sites
        lqcd.lqcd_spinor_gaussian(ctx, Lc, lqcd.field(full_d, lqcd.LQCD_LAYOUT_EO), lqcd.LQCD_EVEN, 7, 0)
        n_half, _ = lqcd.field_bytes(Lc, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
        phi_d = full_d[: n_half // 8]  # the even half of the EO field
        x_d = torch.zeros_like(phi_d)
        fphi = lqcd.field(phi_d, lqcd.LQCD_LAYOUT_EO)
        xc = lqcd.field(x_d, lqcd.LQCD_LAYOUT_EO)
        lqcd.lqcd_fermion_force(ctx, G, fphi, F, kappa, mu, cg, X_cache=xc)
        tff, _ = _timed(torch, lambda: lqcd.lqcd_fermion_force(ctx, G, fphi, F, kappa, mu, cg, X_cache=xc), 5)
        tpl, _ = _timed(torch, lambda: lqcd.lqcd_plaquette(ctx, G), 5)
        misc = {"fermion_force_ms": 1e3 * tff,
                "fermion_force_GBs_paper_count": 4 * Vc * 4736 / tff / 1e9,
                "plaquette_ms": 1e3 * tpl}
        config_line("HMC setup C", None,
                    {"s_per_trajectory": statistics.median(secs),
                     "dH": [s["dH"] for s in trajs], "accepted": [s["accepted"] for s in trajs],
                     "acceptance": sum(s["accepted"] for s in trajs) / len(trajs),
                     "cg_iters_per_trajectory": [s["cg_iters"] for s in trajs],
                     "exp_minus_dH_mean": float(np.mean([np.exp(-s["dH"]) for s in trajs])),
                     "plaquette": [s["plaquette"] for s in trajs], "plaquette_after_heatbath": plaq0,
                     "heatbath_s": thb, "thermalisation_trajectories": len(therm),
                     "thermalisation_dH": [s["dH"] for s in therm],
                     "thermalisation_plaquette": [s["plaquette"] for s in therm],
                     "gauge_force_ms": gf, "force_prec": args.force_prec, "kernels": misc},
                    {"workload": "24^3x8, tlSym beta=3.9, kappa=0.160856, a mu=0.1, 2MN 10 fermion x 10 "
                                 f"gauge steps, tau=1, {args.force_prec} gauge force, F32-inner/DF64 CG to "
                                 "1e-10 per force; start: "
                                 f"{min(args.sweeps, 100)} Wilson heatbath sweeps at beta=6.0 from cold"})
    elif c == "hb":
        # heatbath and overrelaxation throughput (Sec. 5.1) in FP64, counted with the
        # paper's per-link flop figures (Table "rw_flops": 3912 heatbath, 3846 overrelax)
        res = {}
        for Lc in ((16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 32), (32, 32, 32, 64)):
            V = int(np.prod(Lc))
            G = lqcd.lqcd_gauge_import(ctx, torch.from_numpy(inputs.random_gauge(Lc, "cold")).cuda(), Lc,
                                       recon=18)
            for s_ in range(5):
                lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 9, s_)
            row = {}
            for pn in ("f64", "df64", "f32"):
                pr = PREC_NAMES[pn]
                th, _ = _timed(torch, lambda: lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 9, 100, prec=pr), 5)
                tho, _ = _timed(torch, lambda: lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 9, 101, n_or=4, prec=pr), 5)
                tor = (tho - th) / 4
                row[pn] = {"heatbath_ms": 1e3 * th, "overrelax_ms": 1e3 * tor,
                           "heatbath_GFLOPs": 4 * V * 3912 / th / 1e9,
                           "overrelax_GFLOPs": 4 * V * 3846 / tor / 1e9,
                           "heatbath_GBs_paper_count": 4 * V * 2880 / th / 1e9}
            row["plaquette"] = lqcd.lqcd_plaquette(ctx, G)
            res["x".join(map(str, Lc))] = row
            G.free()
        config_line("heatbath", None, {"hb": res},
                    {"workload": "Cabibbo-Marinari heatbath and overrelaxation sweeps, FP64, FP64 with "
                                 "float-float staples (df64) and FP32 (FP32 times include the write-back "
                                 "into the FP64 field), beta=5.7, "
                                 "GFLOP/s with the paper's 3912 / 3846 flop per link"})
    elif c == "hop12":
        # the multi-RHS half hop (12 RHS; F32 with REC12 and 18-real links, or
        # --prec bf16s / f16s with REC12) against the single-RHS hop on 24^3 x 48
        # and 32^3 x 64 near-identity fields; the 12-RHS REC12 launches of the
        # last lattice run inside the NVTX range "hop_multi"
        res = {}
        hp = PREC_NAMES[args.prec] if args.prec in ("bf16s", "f16s") else lqcd.LQCD_F32
        for Lc in ((32, 32, 32, 64), (24, 24, 24, 48)):
            U = torch.from_numpy(inputs.random_gauge(Lc, "near", seed=4100, eps=0.3)).cuda()
            for recon in ((12, 18) if hp == lqcd.LQCD_F32 else (12,)):
                G = lqcd.lqcd_gauge_import(ctx, U, Lc, recon=recon)
                one = time_half_hop_L(ctx, G, lqcd, torch, Lc, hp)
                multi = time_hop_multi(ctx, G, lqcd, torch, Lc, 12, prec=hp,
                                       nvtx=(Lc[0] == 24 and recon == 12))
                res[f"{'x'.join(map(str, Lc))}/rec{recon}"] = {
                    "single_ms": one["ms"], "single_GBs": one["gbs"], "multi12_ms": multi["ms"],
                    "multi12_GBs": multi["gbs"], "multi12_pct_hbm": 100 * multi["gbs"] / peaks["hbm_gbs"],
                    "speedup_vs_12_single": 12 * one["ms"] / multi["ms"],
                    "bytes_per_rhs_site": multi["bytes_per_rhs_site"]}
                G.free()
        config_line("multi-RHS hop", None, {"hop": res},
                    {"workload": f"{[k for k, v in PREC_NAMES.items() if v == hp][0]} half hop, 12 right-hand "
                                 "sides vs one, 24^3x48 and 32^3x64, exp(i 0.3 H) links"})
    elif c == "mrhs":
        # the default line's 12-RHS solve alone (24^3 x 48 bench field, 12 point
        # sources, float-float outer / FP32 inner): one warm-up solve, then one
        # solve inside the NVTX range "mrhs_solve" and one 12-RHS half hop
        U = torch.from_numpy(make_inputs()[0]).cuda()
        G = lqcd.lqcd_gauge_import(ctx, U, L, recon=18)
        b12 = inputs.point_sources(L)
        prm = lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32, max_iter=50000,
                             sloppy_recon=12, check_every=20)
        bd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, 12)
        xd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64, 12)
        fb = lqcd.field(bd, lqcd.LQCD_LAYOUT_EO, nrhs=12)
        fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO, nrhs=12)
        lqcd.lqcd_spinor_pack(ctx, L, torch.from_numpy(b12).cuda(), fb)
        lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm)
        lqcd.lib().lqcd_reset_counters(ctx.handle)
        nvtx_push("mrhs_solve")
        t, st = _timed(torch, lambda: lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm))
        nvtx_pop()
        cnt = lqcd.lqcd_counters()
        lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
        config_line("12-RHS solve", None,
                    {"solve_s": t, "iters_max": max(s["iters"] for s in st),
                     "reliable_updates": max(s["reliable_updates"] for s in st),
                     "true_resid_max": max(s["true_resid"] for s in st), "launches": int(cnt.launches)},
                    {"workload": "24^3x48 exp(i 0.3 H) links, 12 point sources, DF64 outer / F32 inner, "
                                 "REC12 sloppy links, 1e-10"})
    elif c == "dd":
        # the domain-decomposed CG (t split into nt domains held in one
        # process, faces moved by device copies), FP64 and with an F32 or
        # float-float inner solve (defect correction), against lqcd_cg_solve
        # on the default 24^3 x 48 workload: the cost of the decomposition
        # itself (face packs, split hops, one host synchronisation per norm)
        from paper_1209_5942_gb300 import dd
        U, b = make_inputs()
        G = lqcd.lqcd_gauge_import(ctx, torch.from_numpy(U).cuda(), L, recon=18)
        prm = lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_F64, max_iter=50000)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        fb, fx = lqcd.field(bd, lqcd.LQCD_LAYOUT_LEXI), lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI)
        lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm)
        t1, st1 = _timed(torch, lambda: lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm))
        res = {"single_domain": {"solve_s": t1, "iters": st1[0]["iters"], "true_resid": st1[0]["true_resid"]}}
        prm_m = lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_F64, inner_prec=lqcd.LQCD_F32, max_iter=50000)
        lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm_m)
        tm, stm = _timed(torch, lambda: lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm_m))
        res["single_domain_f64/f32"] = {"solve_s": tm, "iters": stm[0]["iters"],
                                        "true_resid": stm[0]["true_resid"]}
        hop_single = {pn: time_hop_multi(ctx, G, lqcd, torch, L, 1, PREC_NAMES[pn], reps=20)
                      for pn in ("f64", "df64", "f32")}
        G.free()
        dd_prms = {"f64": prm,
                   "f64/f32": lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_F64, inner_prec=lqcd.LQCD_F32,
                                             max_iter=50000, max_restarts=10),
                   "f64/df64": lqcd.cg_params(tol=TOL, outer_prec=lqcd.LQCD_F64, inner_prec=lqcd.LQCD_DF64,
                                              max_iter=50000)}
        for nz, nt in ((1, 1), (1, 2), (1, 4), (2, 2)):
            slabs = dd.DomainGrid(L, nz, nt)
            Ll = slabs.local_L
            gs, bs, xs, keep = [], [], [], []
            for d in range(slabs.ndomains):
                gs.append(lqcd.lqcd_gauge_import(ctx, torch.from_numpy(U[slabs.block(d)]).cuda(), Ll, recon=18,
                                                 antiperiodic_t=False))
                bdd, _ = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, lqcd.LQCD_F64)
                xdd, _ = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, lqcd.LQCD_F64)
                f = lqcd.field(bdd, lqcd.LQCD_LAYOUT_EO)
                lqcd.lqcd_spinor_pack(ctx, Ll, torch.from_numpy(b[slabs.block(d)]).cuda(), f, antiperiodic_t=False)
                bs.append(f)
                xs.append(lqcd.field(xdd, lqcd.LQCD_LAYOUT_EO))
                keep.append((bdd, xdd))
            faces = [dd.domain_faces(slabs, lqcd.LQCD_F64) for _ in range(slabs.ndomains)]
            for name, pv in dd_prms.items():
                dd.cg_solve_local_domains(ctx, slabs, gs, bs, xs, KAPPA, MU, pv, faces=faces)
                t, st = _timed(torch, lambda: dd.cg_solve_local_domains(ctx, slabs, gs, bs, xs, KAPPA, MU, pv,
                                                                        faces=faces))
                grid = f"nt{nt}" if nz == 1 else f"nz{nz}nt{nt}"
                key = grid if name == "f64" else f"{grid}_{name}"
                res[key] = {"solve_s": t, "iters": st["iters"], "restarts": st["restarts"],
                            "true_resid": st["true_resid"], "vs_single_domain": t / t1}
            if nt > 1:  # the domain kernels alone, against the undivided lattice's hop
                for pn in ("f64", "df64", "f32"):
                    k = time_dd_kernels(ctx, dd, slabs, gs, lqcd, torch, PREC_NAMES[pn], label=f"dd_hops_{grid}_{pn}")
                    k["hop_pct_hbm"] = 100 * k["hop_GBs"] / peaks["hbm_gbs"]
                    k["single_domain_hop_ms"] = hop_single[pn]["ms"]
                    res[f"{grid}_kernels_{pn}"] = k
            for G_ in gs:
                G_.free()
        config_line("domain-decomposed CG", None, {"dd": res},
                    {"workload": "24^3x48 exp(i 0.3 H) links, kappa=0.16, 2 kappa mu=0.005, CG to 1e-10 "
                                 "(FP64, or FP64 outer with an F32 / float-float inner solve); "
                                 "t split into nt domains (nz x nt: z and t) on one GPU (faces by device copies)"})
    elif c == "sweep":
        res = {}
        for ns in (16, 24, 32, 48):
            for nt in (4, 8, 12, 16):
                Lc = (ns, ns, ns, nt)
                U = torch.from_numpy(inputs.random_gauge(Lc, "near", seed=7000 + ns + nt, eps=0.3)).cuda()
                G = {18: lqcd.lqcd_gauge_import(ctx, U, Lc, recon=18),
                     12: lqcd.lqcd_gauge_import(ctx, U, Lc, recon=12)}
                row = {}
                for pname, prec, recon in (("f64", 0, 18), ("df64", 1, 18), ("f32", 2, 12),
                                           ("bf16s", 3, 12)):
                    h = time_half_hop_L(ctx, G[recon], lqcd, torch, Lc, prec)
                    row[pname + f"/rec{recon}"] = {"GBs": h["gbs"],
                                                   "pct_hbm": 100 * h["gbs"] / peaks["hbm_gbs"],
                                                   "GFLOPs": 1e3 * h["tflops"]}
                res[f"{ns}^3x{nt}"] = row
                G[18].free()
                G[12].free()
        config_line("Dslash sweep", None, {"hop": res},
                    {"workload": "half hop on Ns^3 x Nt, Ns in 16,24,32,48, Nt in 4,8,12,16 "
                                 "(the paper's lattice range), exp(i 0.3 H) links"})


def time_half_hop_L(ctx, G, lqcd, torch, Lc, prec, reps=20):
    n_half, sb = lqcd.field_bytes(Lc, lqcd.LQCD_EVEN, prec, 1)
    din = torch.zeros(n_half // 8, dtype=torch.float64, device="cuda")
    dout = torch.zeros_like(din)
    s_in = torch.ones(max(sb // 4, 1), dtype=torch.float32, device="cuda") if sb else None
    s_out = torch.zeros_like(s_in) if sb else None
    fi = lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec, 1, s_in)
    fo = lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec, 1, s_out)
    lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    t, _ = _timed(torch, lambda: lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0), reps)
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    return {"ms": 1e3 * t, "gbs": cnt.hop_bytes / reps / t / 1e9, "tflops": cnt.hop_flops / reps / t / 1e12}


def time_dd_kernels(ctx, dd, slabs, gauges, lqcd, torch, prec, reps=20, label=None):
    """The domain-decomposed half hop's kernels on every domain of `slabs`
    (one device): the domain hops alone (the faces already in place) and the
    face packs alone, each timed with CUDA events over `reps` half hops;
    GB/s from the library's counted algorithmic bytes.  label: the timed hops
    run inside the NVTX range "<label>" (for an ncu capture of that launch)."""
    Ll = slabs.local_L
    n_half, _ = lqcd.field_bytes(Ll, lqcd.LQCD_EVEN, prec, 1)
    gen = torch.Generator(device="cuda").manual_seed(13)
    keep, ins, outs = [], [], []
    for _ in range(slabs.ndomains):
        din = torch.randn(n_half // 4, dtype=torch.float32, device="cuda", generator=gen).view(torch.float64)
        dout = torch.zeros_like(din)
        keep.append((din, dout))
        ins.append(lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec))
        outs.append(lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec))
    faces = [dd.domain_faces(slabs, prec) for _ in range(slabs.ndomains)]
    dd.dslash_local_domains(ctx, slabs, gauges, ins, outs, lqcd.LQCD_EVEN, 0, bufs=faces)

    def hops():
        for d in range(slabs.ndomains):
            z = faces[d][6:8] if slabs.nz > 1 else (None, None)
            lqcd.lqcd_dd_dslash_zt(ctx, gauges[d], ins[d], outs[d], faces[d][2], faces[d][3], z[0], z[1],
                                   lqcd.LQCD_EVEN, 0)

    def packs():
        for d in range(slabs.ndomains):
            for k, mu in enumerate(slabs.dirs):
                lqcd.lqcd_dd_pack_dir(ctx, gauges[d], ins[d], mu, faces[d][4 * k], faces[d][4 * k + 1],
                                      lqcd.LQCD_EVEN, 0, slabs.negate_to_prev(d, mu), slabs.negate_to_next(d, mu))

    out = {}
    for name, fn in (("hop", hops), ("pack", packs)):
        fn()
        torch.cuda.synchronize()
        c0, c1 = lqcd.lqcd_counters(), lqcd.lqcd_counters()
        lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(c0))
        if label and name == "hop":
            nvtx_push(label)
        t, _ = _timed(torch, fn, reps)
        if label and name == "hop":
            nvtx_pop()
        lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(c1))
        out[f"{name}_ms"] = 1e3 * t
        out[f"{name}_GBs"] = (c1.bytes - c0.bytes) / reps / t / 1e9
    return out


def time_hop_multi(ctx, G, lqcd, torch, Lc, nrhs, prec=2, reps=10, nvtx=False):
    """Multi-RHS half hop: counted bytes read each link once for all RHS."""
    n_half, sb = lqcd.field_bytes(Lc, lqcd.LQCD_EVEN, prec, nrhs)
    gen = torch.Generator(device="cuda").manual_seed(11)
    din = torch.randn(n_half // 4, dtype=torch.float32, device="cuda", generator=gen)
    if sb:  # 16-bit formats: finite stored values below 1, unit site scales
        din = (din.view(torch.int32) & 0x3F7F3F7F).view(torch.float32)
    din = din.view(torch.float64)
    dout = torch.zeros_like(din)
    s_in = torch.ones(max(sb // 4, 1), dtype=torch.float32, device="cuda") if sb else None
    s_out = torch.zeros_like(s_in) if sb else None
    fi = lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec, nrhs, s_in)
    fo = lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec, nrhs, s_out)
    lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    if nvtx:  # ncu --nvtx --nvtx-include hop_multi/ captures these launches
        nvtx_push("hop_multi")
    t, _ = _timed(torch, lambda: lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0), reps)
    if nvtx:
        nvtx_pop()
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    per_rhs_site = cnt.hop_bytes / reps / cnt.hop_sites * reps
    return {"ms": 1e3 * t, "gbs": cnt.hop_bytes / reps / t / 1e9, "nrhs": nrhs, "prec": prec,
            "bytes_per_rhs_site": per_rhs_site}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f64", choices=list(PREC_NAMES))
    ap.add_argument("--inner", default=None, choices=list(PREC_NAMES))
    ap.add_argument("--recon", type=int, default=18)
    ap.add_argument("--check-every", type=int, default=20)
    ap.add_argument("--ref-iters", type=int, default=5)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the half hop, if captured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action="store_true", help="also BiCGStab variants")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the precision variants and the 12-RHS comparison")
    ap.add_argument("--config", default="2", choices=["1", "2", "3", "4a", "4b", "5", "C", "hb", "sweep", "hop12", "mrhs",
                                                     "dd"],
                    help="2 (default): the 24^3x48 contract line; others print their own line")
    ap.add_argument("--sweeps", type=int, default=200, help="heatbath sweeps for configs 3, 4a, 5")
    ap.add_argument("--trajs", type=int, default=10, help="measured HMC trajectories for config 5")
    ap.add_argument("--therm", type=int, default=20, help="HMC thermalisation trajectories for config 5")
    ap.add_argument("--quick", action="store_true", help="config 4a: 2 sequential solves, scaled")
    ap.add_argument("--force-prec", default="df64", choices=["f64", "df64"],
                    help="config C: arithmetic of the gauge force (H and dH are FP64 either way)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config != "2":
        run_config(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

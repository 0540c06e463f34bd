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
           stream; FP64 arithmetic is bound by the FP64 pipe (bound "alu"),
           float-float and lower precisions by HBM
  e2e      the same metric through the public API with host buffers: links
           and source copied host->device, gauge import, solve, solution
           copied device->host, all inside the timed region
  cpu_baseline  the FP64 oracle (C + OpenMP) running a bounded number of CG
           iterations of the same system on the host cores

--impl reference times the oracle itself on the same workload (the paper has
no runnable reference implementation).  --gpus N > 1 runs N independent
replicas (the solve does not shard across GPUs in this build).
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
# FP64 peak of the FP64 pipe: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
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
    G = lqcd.lqcd_gauge_import(ctx, U_d, L, recon=recon)
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
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step()[0])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes_byref(cnt))
    t_local = ms / 1e3
    t = t_local
    bytes_local = cnt.bytes
    if dist:
        tt = torch.tensor([t_local], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
        bb = torch.tensor([bytes_local], device="cuda", dtype=torch.float64)
        dist.all_reduce(bb, op=dist.ReduceOp.SUM)
        bytes_total = float(bb.item())
    else:
        bytes_total = bytes_local
    value = bytes_total / t / 1e9

    # dominant kernel: the half hop of the solve, timed alone on the library stream
    hop = time_half_hop(ctx, G, lqcd, torch, inner, recon, stream)

    # end to end through the public API with host buffers
    e2e = run_e2e(ctx, lqcd, torch, U_h, b_h, prm, recon, args, stream)

    peaks, peak_kind = measured_peaks()
    if inner == lqcd.LQCD_F64:
        roof = {"bound": "alu", "achieved": hop["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": hop["tflops"] / FP64_PEAK_TFLOPS, "traffic": args.traffic,
                "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                "hbm_GBs": hop["gbs"], "hbm_frac": hop["gbs"] / peaks["hbm_gbs"]}
    else:
        roof = {"bound": "hbm", "achieved": hop["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hop["gbs"] / peaks["hbm_gbs"], "traffic": args.traffic,
                "peak_kind": f"{peak_kind} (copy bandwidth, burst)", "tflops": hop["tflops"]}
    roof["kernel"] = hop["kernel"]
    roof["bytes_per_launch"] = hop["bytes"]
    roof["ms_per_launch"] = hop["ms"]

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
    if rank == 0 and args.variants:
        line["variants"] = run_variants(ctx, G, fb, fx, lqcd, torch, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def ctypes_byref(x):
    import ctypes
    return ctypes.byref(x)


def time_half_hop(ctx, G, lqcd, torch, prec, recon, stream, reps=30):
    """Average duration of the half hop (no epilogue) with CUDA events."""
    n_half, sb = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
    din = torch.zeros(n_half // 8, dtype=torch.float64, device="cuda")
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
    e0.record(stream)
    for _ in range(reps):
        lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
    e1.record(stream)
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
    U_pin = torch.from_numpy(U_h).pin_memory()
    b_pin = torch.from_numpy(b_h).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    U_dev = torch.empty(U_pin.shape, dtype=U_pin.dtype, device="cuda")
    b_dev = torch.empty(b_pin.shape, dtype=b_pin.dtype, device="cuda")
    x_dev = torch.empty_like(b_dev)

    def step():
        U_dev.copy_(U_pin, non_blocking=True)
        b_dev.copy_(b_pin, non_blocking=True)
        G = lqcd.lqcd_gauge_import(ctx, U_dev, L, recon=recon)
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


def run_variants(ctx, G, fb, fx, lqcd, torch, stream):
    """Time-to-1e-10 on the same system for the other precision paths (one warm-up
    solve and one timed solve each)."""
    out = {}
    combos = [("f64", "f64"), ("df64", "df64"), ("df64", "f32"), ("df64", "bf16s"),
              ("df64", "f16s")]
    for outer, inner in combos:
        prm = lqcd.cg_params(tol=TOL, outer_prec=PREC_NAMES[outer], inner_prec=PREC_NAMES[inner],
                             max_iter=50000)
        try:
            lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = lqcd.lqcd_cg_solve(ctx, G, fb, fx, KAPPA, MU, prm)[0]
            dt = time.perf_counter() - t0
            out[f"{outer}/{inner}"] = {"time_to_solution_s": dt, "iters": st["iters"],
                                       "reliable_updates": st["reliable_updates"],
                                       "true_resid": st["true_resid"]}
        except Exception as e:  # report, do not hide
            out[f"{outer}/{inner}"] = {"error": str(e)}
    return out


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
    ap.add_argument("--variants", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

"""Benchmark: MLUPS and HBM-roofline fraction of the fused stream + collide step on one GB300.

Workload (default): D3Q19 anisotropic BGK, FP32 storage, 256^3 fully periodic Taylor-Green vortex
(u0 = 0.02, rho0 = 1), tau = 0.6, Theta = R diag(0.36, 0.33, 0.30) R^T with a seeded rotation R.
One bench step = one lattice time step over the whole 256^3 box = one kernel launch. The
populations (2 x 1.28 GB) exceed the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0). Extra keys: roofline (dominant kernel, CUDA events), cpu_baseline
(the FP64 oracle on a bounded sample), e2e (through the public API with host buffers), clocks,
gpu_launches, and sub-measurements for FP16-shifted storage and the checkpointed adjoint.
`--impl reference` times the oracle itself (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0

# DRAM traffic per launch from an ncu capture, keyed by workload; valid only while the kernel
# source hash matches the one recorded with the counters (else the bench reports null).
NCU_TRAFFIC = {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("lbm_kernels.cuh", "lbm_lattice.cuh", "lbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_27004_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
WORKLOADS = {
    # name: (q, n, storage, tau, description)
    "d3q19_fp32_256": dict(q=19, n=256, storage="fp32", tau=0.6,
                           desc="D3Q19 FP32 256^3 periodic Taylor-Green, rotated Theta, tau 0.6"),
    "d3q19_fp16s_256": dict(q=19, n=256, storage="fp16s", tau=0.6,
                            desc="D3Q19 FP16-shifted 256^3 periodic Taylor-Green"),
}


def bytes_per_cell(q, storage):
    elem = {"fp32": 4, "fp32s": 4, "fp16s": 2, "fp64": 8}[storage]
    return 2 * q * elem


def make_problem(w):
    from paper_2605_27004_gb300 import inputs
    n = w["n"]
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    return Th, rho0, u0


def time_forward(w, steps, warmup, torch, lbm):
    """Device-timed forward steps: returns (ms total, per-launch ms list, launches, ctx)."""
    n, q = w["n"], w["q"]
    Th, rho0, u0 = make_problem(w)
    L = lbm.LBM(q, n, n, n, w["tau"], Th, storage=w["storage"])
    L.init(torch.as_tensor(rho0, dtype=torch.float32), torch.as_tensor(u0, dtype=torch.float32))
    L.step(warmup)
    stream = L.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = L.launches
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        L.step(1)
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = L.launches - l0
    per = [a.elapsed_time(b) for a, b in ev]
    return t0.elapsed_time(t1), per, launches, L


def time_e2e(w, steps, torch, lbm):
    """Public API with host buffers: pinned H2D of (rho0, u0), init, steps, moments, D2H of u."""
    n, q = w["n"], w["q"]
    Th, rho0, u0 = make_problem(w)
    N = n ** 3
    rho_h = torch.as_tensor(rho0, dtype=torch.float32).pin_memory()
    u_h = torch.as_tensor(u0, dtype=torch.float32).reshape(3, N).pin_memory()
    out_h = torch.empty((3, N), dtype=torch.float32).pin_memory()
    L = lbm.LBM(q, n, n, n, w["tau"], Th, storage=w["storage"])
    rho_d = torch.empty(N, dtype=torch.float32, device="cuda")
    u_d = torch.empty((3, N), dtype=torch.float32, device="cuda")
    out_d = torch.empty((3, N), dtype=torch.float32, device="cuda")
    stream = L.stream
    # warm-up of the same sequence
    rho_d.copy_(rho_h, non_blocking=True)
    u_d.copy_(u_h, non_blocking=True)
    L.init(rho_d, u_d)
    L.step(2)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    rho_d.copy_(rho_h, non_blocking=True)
    u_d.copy_(u_h, non_blocking=True)
    L.init(rho_d, u_d)
    L.step(steps)
    L.moments_into(u=out_d)
    out_h.copy_(out_d, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    h2d = (rho_h.numel() + u_h.numel()) * 4
    d2h = out_h.numel() * 4
    L.close()
    return ms, h2d, d2h


def time_adjoint(q, n, storage, steps, K, torch, lbm):
    """Checkpointed adjoint through `steps` steps: ms of lbm_adjoint (recompute + adjoint sweep)."""
    from paper_2605_27004_gb300 import inputs
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    L = lbm.LBM(q, n, n, n, 0.6, Th, storage=storage)
    L.init(torch.as_tensor(rho0, dtype=torch.float32), torch.as_tensor(u0, dtype=torch.float32))
    L.step(steps)
    g = torch.randn(3, n ** 3, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    t = time.perf_counter()
    L.adjoint(g, steps, K)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) * 1e3
    L.close()
    return ms


def cpu_baseline(w, budget_s=12.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload: a 64^3 sub-box of the
    same Taylor-Green problem, as many steps as fit the budget."""
    import oracle
    from paper_2605_27004_gb300 import inputs
    n = 64
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    pb = oracle.Problem(w["q"], n, n, n, w["tau"], Th)
    f = pb.init(rho0, u0)
    t = time.perf_counter()
    pb.run(f, 1)
    one = time.perf_counter() - t
    steps = max(1, int(budget_s / max(one, 1e-3)))
    t = time.perf_counter()
    pb.run(f, steps)
    dt = time.perf_counter() - t
    return {"value": n ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{w['desc'].split(' 256^3')[0]} on a 64^3 box, {steps} steps, FP64 push oracle"}


def run_reference(args):
    """Reference arm: the oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    import oracle
    from paper_2605_27004_gb300 import inputs
    n = 64
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    pb = oracle.Problem(w["q"], n, n, n, w["tau"], Th)
    f = pb.init(rho0, u0)
    pb.run(f, max(1, args.warmup))
    t = time.perf_counter()
    pb.run(f, args.steps)
    dt = time.perf_counter() - t
    v = n ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["desc"] + " (oracle sample: 64^3 box)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"64^3 box of the workload, {args.steps} timed steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="d3q19_fp32_256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip sub-measurements, e2e and cpu baseline")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOADS[args.workload]
    n, q = w["n"], w["q"]
    N = n ** 3

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # cpu baseline first (host only, before the timed GPU region)
    cpu = cpu_baseline(w) if (rank == 0 and world == 1 and not args.no_extras) else None

    barrier()
    with ClockSampler(local) as clk:
        ms, per, launches, L = time_forward(w, args.steps, args.warmup, torch, lbm)
    barrier()
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    mlups = N * args.steps * world / (ms * 1e-3) / 1e6
    peak, peak_src = measured_peak()
    bpc = bytes_per_cell(q, w["storage"])
    kern_ms = float(np.mean(per))
    achieved = bpc * N / (kern_ms * 1e-3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get(args.workload)
    if rec and rec.get("kernel_sha") == kernel_source_hash():
        traffic = rec["traffic_bytes"]
    L.close()
    del L
    torch.cuda.empty_cache()

    sub = {}
    e2e = None
    if not args.no_extras:
        if rank == 0:
            wf = WORKLOADS["d3q19_fp16s_256"]
            ms16, per16, _, L16 = time_forward(wf, max(10, args.steps // 2), args.warmup, torch, lbm)
            L16.close()
            k16 = float(np.mean(per16))
            sub["fwd_fp16s_256"] = {"mlups": N * len(per16) / (ms16 * 1e-3) / 1e6,
                                    "kernel_gbs": bytes_per_cell(19, "fp16s") * N / (k16 * 1e-3) / 1e9,
                                    "frac": bytes_per_cell(19, "fp16s") * N / (k16 * 1e-3) / 1e9 / peak}
            nadj, Kadj, nA = 200, 20, 128
            msa = time_adjoint(19, nA, "fp32", nadj, Kadj, torch, lbm)
            sub["adjoint_fp32_128"] = {"mlups": nA ** 3 * nadj / (msa * 1e-3) / 1e6, "steps": nadj,
                                       "checkpoint_every": Kadj,
                                       "note": "wall time of lbm_adjoint incl. forward recompute"}
        msE, h2d, d2h = time_e2e(w, args.steps, torch, lbm)
        e2e = {"value": N * args.steps * world / (msE * 1e-3) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "one upload of (rho0, u0), init, K steps, moments, one download of u; bytes amortised per step"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "cells": N, "lattice": f"D3Q{q}", "storage": w["storage"],
                   "l2": "inputs larger than L2 (2 x %.2f GB populations)" % (q * N * 4 / 1e9),
                   "parallelism": "independent replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "kernel": "k_step_pull<19, FP32>", "bytes_per_cell": bpc,
                     "kernel_ms_mean": kern_ms},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "sub": sub,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

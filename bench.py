"""Benchmark: MLUPS and HBM-roofline fraction of the fused stream + collide step on one GB300.

Default workload: D3Q19 anisotropic BGK, FP32 storage (the default shifted form f - r_i, FP32
arithmetic), 256^3 fully periodic Taylor-Green vortex
(u0 = 0.02, rho0 = 1), tau = 0.6, Theta = R diag(0.36, 0.33, 0.30) R^T with a seeded rotation R.
One bench step = one lattice time step over the whole box = one kernel launch. The populations
(2 x 1.28 GB) exceed the 129 MB L2, so no flush is needed between steps.

Modes
  (default)   the one-line JSON contract: value = MLUPS of the forward step (device time),
              roofline of the dominant kernel, cpu_baseline (oracle), e2e (public API with host
              buffers), clocks, gpu_launches, plus sub-measurements (FP16-shifted forward, the
              checkpointed adjoint).
  --mode sweep     one JSON line per variant (lattice x storage x scheme x size, porous runs).
  --mode profile   a small case of one kernel for ncu (--lattice/--storage/--scheme/--n/--kernel).
  --mode slabs     the z-slab decomposition on one GPU against the whole box (--n, --storage).
  --mode oracle    the FP64 oracle on a bounded sample of each workload (host cores, no GPU).
  --sharded        the contract line for one box cut into z-slabs over the ranks (strong scaling,
                   halo exchange over torch.distributed) instead of independent replicas.
  --impl reference the oracle itself timed on the host cores (the reference arm).
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
ELEM = {"fp32": 4, "fp32s": 4, "fp16s": 2, "fp16w": 2, "fp64": 8}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the headline kernel from
# one ncu capture of `python bench.py --mode profile --storage fp32s --n 256`, keyed by variant.
# It is used only while the kernel sources hash to the value recorded with the capture; after a
# kernel change the bench reports traffic = null (with the reason) until the capture is redone.
NCU_TRAFFIC = {
    # mean of 3 launches at 256^3: read 1.27521e9 + write 1.22052e9 bytes
    "d3q19_fp32s_pull": {"traffic_bytes": 2.4957e+09, "kernel_sha": "d1d5effa5735a487"},
}


def kernel_source_hash() -> str:
    """Hash of the sources that define the headline kernel (its body, the lattice tables and the
    parameter structs with the block-shape rule)."""
    h = hashlib.sha256()
    for f in ("lbm_kernels.cuh", "lbm_lattice.cuh", "lbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_27004_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def host_mem_available() -> float:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) * 1024.0
    except OSError:
        pass
    return 0.0


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    EXTRA = ",clocks.mem,temperature.gpu,temperature.memory"  # used when this nvidia-smi accepts them

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            fields = self.FIELDS + self.EXTRA
            probe = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={fields}",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            if probe.returncode != 0:
                fields = self.FIELDS
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={fields}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
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
        out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}
        extra = {"mem_mhz": [], "gpu_temp_c": [], "hbm_temp_c": []}
        for line in self.out:  # memory clock and temperatures (N/A on some parts)
            parts = [p.strip() for p in line.split(",")]
            for k, key in zip(range(9, 12), extra):
                try:
                    extra[key].append(float(parts[k]))
                except (ValueError, IndexError):
                    pass
        if extra["mem_mhz"]:
            out["mem_mhz"] = float(np.median(extra["mem_mhz"]))
        for key in ("gpu_temp_c", "hbm_temp_c"):
            if extra[key]:
                out[key + "_max"] = max(extra[key])
        return out


# ------------------------------------------------------------------------------------------------
# Problems
# ------------------------------------------------------------------------------------------------
def theta3():
    from paper_2605_27004_gb300 import inputs
    return inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)


def problem(q, n, kind):
    """(dims, tau, Theta, rho0, u0, solid) of a named synthetic workload at size n."""
    from paper_2605_27004_gb300 import inputs
    if kind == "tg":
        if q == 9:
            rho0, u0 = inputs.taylor_green_2d(n, 0.02)
            return (n, n, 1), 0.8, inputs.theta_from_atilde([[1.0, 0.2], [0.2, 1.0]]), rho0, u0, None
        if n >= 384:  # same field as inputs.taylor_green_3d, built on the device to spare host memory
            import torch
            k = 2 * np.pi / n
            ax = torch.arange(n, device="cuda", dtype=torch.float32) * k
            s, c = torch.sin(ax), torch.cos(ax)
            u0 = torch.zeros((3, n, n, n), device="cuda", dtype=torch.float32)
            u0[0] = 0.02 * s[None, None, :] * c[None, :, None] * c[:, None, None]
            u0[1] = -0.02 * c[None, None, :] * s[None, :, None] * c[:, None, None]
            return (n, n, n), 0.6, theta3(), None, u0.reshape(3, -1), None
        rho0, u0 = inputs.taylor_green_3d(n, 0.02)
        return (n, n, n), 0.6, theta3(), rho0, u0, None
    if kind == "ade":  # scalar blob in the frozen Taylor-Green field (u0 = 0.05), built on the device
        import torch
        k = 2 * np.pi / n
        ax = torch.arange(n, device="cuda", dtype=torch.float32)
        s, c = torch.sin(ax * k), torch.cos(ax * k)
        u = torch.zeros((3, n, n, n), device="cuda", dtype=torch.float32)
        u[0] = 0.05 * s[None, None, :] * c[None, :, None] * c[:, None, None]
        u[1] = -0.05 * c[None, None, :] * s[None, :, None] * c[:, None, None]
        h = (n - 1) / 2
        r2 = (ax[None, None, :] - h) ** 2 + (ax[None, :, None] - h) ** 2 + (ax[:, None, None] - h) ** 2
        phi = 1.0 + 0.5 * torch.exp(-r2 / (2 * (n / 12) ** 2))
        return (n, n, n), 0.6, theta3(), phi.reshape(-1), u.reshape(3, -1), None
    if kind == "ade_porous":  # scalar blob carried by u_x = 0.03 through the porous medium
        import torch
        solid = inputs.porous_spheres(n, n, n, seed=inputs.SEED_BASE + 3)
        fl = torch.as_tensor(1 - solid, dtype=torch.float32, device="cuda")
        u = torch.zeros((3, n ** 3), device="cuda", dtype=torch.float32)
        u[0] = 0.03 * fl
        ax = torch.arange(n, device="cuda", dtype=torch.float32)
        h = (n - 1) / 2
        r2 = (ax[None, None, :] - h) ** 2 + (ax[None, :, None] - h) ** 2 + (ax[:, None, None] - h) ** 2
        phi = 1.0 + 0.5 * torch.exp(-r2 / (2 * (n / 12) ** 2)).reshape(-1) * fl
        return (n, n, n), 0.7, np.diag([0.38, 0.33, 0.29]), phi, u, solid
    if kind == "porous":
        solid = inputs.porous_spheres(n, n, n, seed=inputs.SEED_BASE + 3)
        N = n ** 3
        u0 = np.zeros((3, N), dtype=np.float32)
        u0[0] = 0.03 * (1 - solid)
        return (n, n, n), 0.7, np.diag([0.38, 0.33, 0.29]), np.ones(N, dtype=np.float32), u0, solid
    raise ValueError(kind)


def make_ctx(q, n, storage, scheme, kind, torch, lbm, **kw):
    dims, tau, Th, rho0, u0, solid = problem(q, n, kind)
    dt = torch.float64 if storage == "fp64" else torch.float32
    if kind in ("ade", "ade_porous"):
        L = lbm.ADE(q, *dims, tau, Th, u=u0.to(dt), solid=solid, storage=storage, scheme=scheme, **kw)
        L.init(rho0.to(dt))
        return L, L.N if solid is None else int((solid == 0).sum())
    L = lbm.LBM(q, *dims, tau, Th, solid=solid, storage=storage, scheme=scheme, **kw)
    L.init(None if rho0 is None else torch.as_tensor(rho0, dtype=dt), torch.as_tensor(u0, dtype=dt))
    n_fluid = L.N if solid is None else int((solid == 0).sum())
    return L, n_fluid


def time_steps(L, steps, warmup, torch):
    """Device time of `steps` single-step launches on the context's stream (CUDA events), plus the
    mean per-launch duration from per-step event pairs."""
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
    per = [a.elapsed_time(b) for a, b in ev]
    return t0.elapsed_time(t1), float(np.mean(per)), L.launches - l0


def variant(q, n, storage, scheme, kind, steps, warmup, torch, lbm, peak):
    L, nf = make_ctx(q, n, storage, scheme, kind, torch, lbm, use_graphs=-1)
    ms, kms, launches = time_steps(L, steps, warmup, torch)
    N = L.N
    L.close()
    ade = kind in ("ade", "ade_porous")
    bpc = 2 * q * ELEM[storage] + ((3 if q != 9 else 2) * (8 if storage == "fp64" else 4) if ade else 0)
    alg = nf * bpc + (4 * N if kind in ("porous", "ade_porous") else 0)  # walls: one 4-byte link word per cell
    gbs = alg / (kms * 1e-3) / 1e9
    return {"lattice": f"D{3 if q != 9 else 2}Q{q}", "n": n, "storage": storage, "scheme": scheme, "kind": kind,
            "cells": N, "fluid_cells": nf, "mlups_all": N * steps / (ms * 1e-3) / 1e6,
            "mlups_fluid": nf * steps / (ms * 1e-3) / 1e6, "kernel_ms": kms, "kernel_gbs": gbs,
            "frac": gbs / peak, "bytes_per_fluid_cell": bpc, "launches": launches}


def variant_graphs(q, n, storage, scheme, steps, warmup, torch, lbm, peak):
    """lbm_step(K) as a caller issues it, one call for all K steps: boxes up to 2M cells replay
    CUDA graphs of 16 steps (the library's default), larger ones launch step by step. Device time
    of the call from CUDA events on the context's stream."""
    L, nf = make_ctx(q, n, storage, scheme, "tg", torch, lbm)
    K = 16 * max(1, steps // 16)
    L.step(16 * max(1, warmup))  # the first call captures the graph
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = L.launches
    t0.record(L.stream)
    L.step(K)
    t1.record(L.stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    launches = L.launches - l0
    N = L.N
    L.close()
    bpc = 2 * q * ELEM[storage]
    gbs = N * bpc * K / (ms * 1e-3) / 1e9
    return {"lattice": f"D3Q{q}", "n": n, "storage": storage, "scheme": scheme, "kind": "tg", "via": "lbm_step(K)",
            "graphs": N <= (1 << 21), "steps": K, "cells": N, "mlups_all": N * K / (ms * 1e-3) / 1e6,
            "ms_per_step": ms / K, "kernel_gbs": gbs, "frac": gbs / peak, "launches": launches}


def time_adjoint(q, n, storage, scheme, steps, K, torch, lbm):
    """Wall time of lbm_adjoint through `steps` steps (forward recompute + reverse sweep), in
    steady state: the second of two calls on the same forward run, as in an optimisation loop
    (the first call also allocates and clears the adjoint's working set; its time is returned
    too). Returns (ms, N, launches, ms_first, plan)."""
    L, nf = make_ctx(q, n, storage, scheme, "tg", torch, lbm)
    L.record_checkpoints(K)  # the forward run keeps the checkpoints the adjoint starts from
    L.step(steps)
    g = torch.randn(3, L.N, device="cuda", dtype=torch.float64 if storage == "fp64" else torch.float32)
    times = []
    for _ in range(2):
        torch.cuda.synchronize()
        l0 = L.launches
        t = time.perf_counter()
        L.adjoint(g, steps, K)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t) * 1e3)
        launches = L.launches - l0
    k2, prefetched = L.adjoint_info()
    N = L.N
    L.close()
    return times[1], N, launches, times[0], {"sub_segment": k2, "host_checkpoints_prefetched": prefetched}


def time_e2e(q, n, storage, steps, torch, lbm):
    """Public API with host buffers: pinned H2D of (rho0, u0), init, steps, moments, D2H of u."""
    dims, tau, Th, rho0, u0, solid = problem(q, n, "tg")
    N = int(np.prod(dims))
    d = 3 if q != 9 else 2
    rho_h = torch.as_tensor(rho0, dtype=torch.float32).pin_memory()
    u_h = torch.as_tensor(u0, dtype=torch.float32).reshape(d, N).pin_memory()
    out_h = torch.empty((d, N), dtype=torch.float32).pin_memory()
    L = lbm.LBM(q, *dims, tau, Th, storage=storage)
    rho_d = torch.empty(N, dtype=torch.float32, device="cuda")
    u_d = torch.empty((d, N), dtype=torch.float32, device="cuda")
    out_d = torch.empty((d, N), dtype=torch.float32, device="cuda")
    stream = L.stream

    def job(k):
        rho_d.copy_(rho_h, non_blocking=True)
        u_d.copy_(u_h, non_blocking=True)
        L.init(rho_d, u_d)
        L.step(k)
        L.moments_into(u=out_d)
        out_h.copy_(out_d, non_blocking=True)

    job(3)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    job(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    L.close()
    return ms, (rho_h.numel() + u_h.numel()) * 4, out_h.numel() * 4


def cpu_baseline(budget_s=12.0):
    """The FP64 oracle as it stands on a bounded sample of the default workload: a 64^3 box of the
    same Taylor-Green problem, as many steps as fit the budget."""
    import oracle
    dims, tau, Th, rho0, u0, _ = problem(19, 64, "tg")
    pb = oracle.Problem(19, *dims, tau, Th)
    f = pb.init(rho0, u0)
    t = time.perf_counter()
    pb.run(f, 1)
    one = time.perf_counter() - t
    steps = max(1, int(budget_s / max(one, 1e-3)))
    t = time.perf_counter()
    pb.run(f, steps)
    dt = time.perf_counter() - t
    return {"value": 64 ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"D3Q19 Taylor-Green on a 64^3 box, {steps} steps of the FP64 push oracle"}


def _timed_oracle_steps(pb, f, budget_s):
    """As many steps of the oracle on f as fit the budget (one step timed first); (steps, s)."""
    t = time.perf_counter()
    pb.run(f, 1)
    one = time.perf_counter() - t
    steps = max(1, int(budget_s / max(one, 1e-4)))
    t = time.perf_counter()
    pb.run(f, steps)
    return steps, time.perf_counter() - t


def oracle_per_config(budget_s=8.0):
    """The FP64 oracle as it stands, on a bounded sample of each workload: rows of
    (config, MLUPS, sample). Forward samples count every cell updated; the adjoint sample counts
    adjoint time steps (the oracle keeps all states and runs its own forward pass)."""
    import oracle
    from paper_2605_27004_gb300 import inputs
    rows = []
    rho0, u0 = inputs.shear_wave_2d(64, 64, 0.01, 1e-4)
    pb = oracle.Problem(9, 64, 64, 1, 0.8, np.array([[0.36, 0.02], [0.02, 0.30]]))
    steps, dt = _timed_oracle_steps(pb, pb.init(rho0, u0), budget_s)
    rows.append(("1 D2Q9 FP64 64^2 shear wave", 64 * 64 * steps / dt / 1e6, f"the full 64^2 box, {steps} steps"))
    dims, tau, Th, rho0, u0, _ = problem(19, 64, "tg")
    pb = oracle.Problem(19, *dims, tau, Th)
    steps, dt = _timed_oracle_steps(pb, pb.init(rho0, u0), budget_s)
    rows.append(("2 D3Q19 Taylor-Green", 64 ** 3 * steps / dt / 1e6, f"a 64^3 box, {steps} steps"))
    dims, tau, Th, rho0, u0, solid = problem(27, 64, "porous")
    pb = oracle.Problem(27, *dims, tau, Th, solid=solid)
    steps, dt = _timed_oracle_steps(pb, pb.init(rho0, u0), budget_s)
    nf = int((np.asarray(solid) == 0).sum())
    rows.append(("3 D3Q27 porous, walls", nf * steps / dt / 1e6,
                 f"a 64^3 porous box of the same recipe ({nf} fluid cells), {steps} steps, fluid-cell MLUPS"))
    _, u0 = inputs.random_fourier_modes(32, 4.0, 0.02)
    pb = oracle.Problem(19, 32, 32, 32, 0.6, np.eye(3) / 3)
    g = np.random.default_rng(inputs.SEED_BASE + 4).standard_normal((3, 32 ** 3))
    t = time.perf_counter()
    pb.adjoint(np.ones(32 ** 3), u0, 2, g)
    one = (time.perf_counter() - t) / 2
    steps = max(2, int(budget_s / max(one, 1e-4)))
    t = time.perf_counter()
    pb.adjoint(np.ones(32 ** 3), u0, steps, g)
    dt = time.perf_counter() - t
    rows.append(("4 D3Q19 adjoint (forward pass, all states kept, reverse sweep)", 32 ** 3 * steps / dt / 1e6,
                 f"a 32^3 box, {steps} adjoint steps"))
    return rows


def job_throughput(ms_local, cells, steps, dist, torch, device="cuda"):
    """Whole-job throughput of independent replicas (one per rank): the slowest rank's time (MAX
    over ranks) and the cells all ranks updated, cells x steps x world size, per second in MLUPS.
    Returns (ms, mlups)."""
    world = 1
    ms = float(ms_local)
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, cells * steps * world / (ms * 1e-3) / 1e6


# ------------------------------------------------------------------------------------------------
def run_reference(args):
    """Reference arm: the oracle, as it stands, timed on the host cores (rank 0 only)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    dims, tau, Th, rho0, u0, _ = problem(19, 64, "tg")
    pb = oracle.Problem(19, *dims, tau, Th)
    f = pb.init(rho0, u0)
    pb.run(f, max(1, args.warmup))
    t = time.perf_counter()
    pb.run(f, args.steps)
    dt = time.perf_counter() - t
    v = 64 ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "D3Q19 256^3 periodic Taylor-Green, rotated Theta, tau 0.6 "
                                   "(each oracle step: a 64^3 box of it)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"64^3 box of the workload, {args.steps} timed FP64 oracle steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args, torch, lbm):
    peak, src = measured_peak()
    cases = []
    for n in (64, 128, 256, 512):
        cases += [(19, n, "fp32s", "pull", "tg"), (19, n, "fp16s", "pull", "tg"), (19, n, "fp16s", "aa", "tg")]
    cases += [(19, 768, "fp16s", "aa", "tg")]
    cases += [(27, 256, "fp32s", "pull", "tg"), (27, 256, "fp16s", "pull", "tg"), (27, 256, "fp16s", "aa", "tg"),
              (19, 256, "fp32s", "aa", "tg"),
              (19, 256, "fp32", "pull", "tg"), (9, 4096, "fp32s", "pull", "tg"), (9, 64, "fp64", "pull", "tg")]
    cases += [(27, 512, "fp32s", "pull", "porous"), (27, 512, "fp16s", "pull", "porous"),
              (27, 512, "fp16s", "aa", "porous")]
    cases += [(19, 256, "fp32s", "pull", "ade"), (19, 256, "fp16s", "pull", "ade"), (19, 256, "fp16s", "aa", "ade"),
              (27, 256, "fp32s", "pull", "ade"), (19, 512, "fp32s", "pull", "ade"),
              (19, 512, "fp32s", "pull", "ade_porous"), (19, 512, "fp16s", "pull", "ade_porous"),
              (27, 256, "fp32s", "pull", "ade_porous")]
    if args.only:
        cases = [c for c in cases if args.only in "%s_%d_%s_%s_%s" % (c[0], c[1], c[2], c[3], c[4])]
    for c in cases:
        q, n, st, sc, kind = c
        try:
            with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
                r = variant(q, n, st, sc, kind, args.steps, args.warmup, torch, lbm, peak)
            r["peak"] = peak
            r["peak_source"] = src
            r["clocks"] = clk.summary()
        except Exception as e:  # report and continue (e.g. memory)
            r = {"case": c, "error": str(e)[:200]}
        print(json.dumps(r), flush=True)
        torch.cuda.empty_cache()
    for (q, n, st, sc) in [(19, 64, "fp32s", "pull"), (19, 64, "fp16s", "pull"), (19, 64, "fp16s", "aa"),
                           (19, 128, "fp32s", "pull"), (19, 128, "fp16s", "pull"), (19, 128, "fp16s", "aa")]:
        if args.only and args.only not in "graphs_%d_%d_%s_%s" % (q, n, st, sc):
            continue
        try:
            r = variant_graphs(q, n, st, sc, max(args.steps, 64), args.warmup, torch, lbm, peak)
            r["peak"] = peak
        except Exception as e:
            r = {"graphs": True, "case": [q, n, st, sc], "error": str(e)[:200]}
        print(json.dumps(r), flush=True)
    # 768^3 first: run after the 512^3 case in the same process (whose host checkpoints were
    # allocated and freed) it measured 0.66 instead of 0.71 of the copy peak, the cause not found
    for (q, n, st, sc, K, steps) in [(19, 768, "fp16s", "aa", 20, 200),
                                     (19, 64, "fp32s", "pull", 20, 200), (19, 64, "fp16s", "aa", 20, 200),
                                     (19, 128, "fp32s", "pull", 20, 200), (19, 128, "fp16s", "pull", 20, 200),
                                     (19, 256, "fp32s", "pull", 20, 100), (19, 256, "fp16s", "aa", 20, 100),
                                     (19, 512, "fp16s", "aa", 20, 200)]:
        if args.only and args.only not in "adj_%d_%d_%s_%s" % (q, n, st, sc):
            continue
        # checkpoints beyond device memory go to pinned host memory: check there is room
        need_host = (steps // K) * q * n ** 3 * ELEM[st]
        if n >= 512 and host_mem_available() < 1.2 * need_host:
            print(json.dumps({"adjoint": True, "lattice": f"D3Q{q}", "n": n, "storage": st, "scheme": sc,
                              "skipped": "host memory %.0f GB < %.0f GB of checkpoints" %
                                         (host_mem_available() / 1e9, 1.2 * need_host / 1e9)}), flush=True)
            continue
        try:
            with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
                ms, N, launches, ms1, plan = time_adjoint(q, n, st, sc, steps, K, torch, lbm)
        except Exception as e:
            print(json.dumps({"adjoint": True, "n": n, "error": str(e)[:300]}), flush=True)
            continue
        bpc = 2 * q * 4 + 3 * q * ELEM[st]  # adjoint kernel (lambda r+w, f_t r) + one recompute step
        mlups = N * steps / (ms * 1e-3) / 1e6
        print(json.dumps({"adjoint": True, "lattice": f"D3Q{q}", "n": n, "storage": st, "scheme": sc, "steps": steps,
                          "checkpoint_every": K, "mlups": mlups, "ms": ms, "bytes_per_cell": bpc,
                          "frac": mlups * 1e6 * bpc / 1e9 / peak, "mlups_first_call": N * steps / (ms1 * 1e-3) / 1e6,
                          "ms_first_call": ms1, "launches": launches, **plan, "clocks": clk.summary()}),
              flush=True)
        torch.cuda.empty_cache()


def run_slabs(args, torch, lbm):
    """The z-slab decomposition on one GPU: the whole n^3 Taylor-Green box (D3Q19) against the same
    box cut into S slabs (one stream and host thread per slab, halo planes exchanged by device
    copies after every step, the host threads meeting at a barrier per exchange), and one slab
    of the one-slab-per-process class at world size 1 (its exchange through the same transport
    function). Wall time over `steps` steps after `warmup`; one JSON line per case."""
    from paper_2605_27004_gb300 import slabs
    n = args.n
    dims, tau, Th, rho0, u0, _ = problem(19, n, "tg")
    N = int(np.prod(dims))
    dt = torch.float64 if args.storage == "fp64" else torch.float32
    r0 = None if rho0 is None else torch.as_tensor(rho0, dtype=dt)
    u0t = torch.as_tensor(u0, dtype=dt) if not isinstance(u0, torch.Tensor) else u0.to(dt)
    for S in (1, 2, 4, 8):
        if S == 1:
            L = lbm.LBM(19, *dims, tau, Th, storage=args.storage, use_graphs=-1)
            L.init(r0, u0t)
            run, close = L.step, L.close
        else:
            G = slabs.SlabGroup(19, *dims, tau, Th, S, storage=args.storage)
            G.init(r0, u0t)
            run, close = G.step, G.close
        run(args.warmup)
        torch.cuda.synchronize()
        t = time.perf_counter()
        run(args.steps)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        close()
        print(json.dumps({"slabs": S, "n": n, "storage": args.storage, "steps": args.steps, "ms_per_step": ms / args.steps,
                          "mlups": N * args.steps / (ms * 1e-3) / 1e6,
                          "case": "whole box" if S == 1 else "SlabGroup, one GPU"}), flush=True)
        torch.cuda.empty_cache()
    D = slabs.DistributedSlab(19, *dims, tau, Th, storage=args.storage)
    D.L.init(None if r0 is None else slabs.slab_of(r0.cuda(), D.plan, dims[0], dims[1]),
             slabs.slab_of(u0t.cuda().reshape(3, -1), D.plan, dims[0], dims[1]))
    ms, kms, _ = time_steps(D.L, args.steps, args.warmup, torch)
    D.L.close()
    print(json.dumps({"slabs": 1, "n": n, "storage": args.storage, "steps": args.steps, "ms_per_step": ms / args.steps,
                      "mlups": N * args.steps / (ms * 1e-3) / 1e6,
                      "case": "DistributedSlab, world size 1 (exchange with itself through the transport)"}),
          flush=True)


def run_sharded(args, torch, lbm, dist, world, rank, local):
    """Strong scaling of the z-slab decomposition: one n^3 D3Q19 Taylor-Green box (default 512^3,
    shifted FP32) cut into `world` slabs, one per rank, the halo planes exchanged over
    torch.distributed (NCCL) after every step. value = cells of the whole box x steps / the
    slowest rank's time. With one rank the slab exchanges with itself through the same code."""
    from paper_2605_27004_gb300 import slabs
    peak, peak_src = measured_peak()
    n = args.n if args.n != 128 else 512
    dims, tau, Th, rho0, u0, _ = problem(19, n, "tg")
    N = int(np.prod(dims))
    D = slabs.DistributedSlab(19, *dims, tau, Th, storage="fp32s")
    u0t = u0 if isinstance(u0, torch.Tensor) else torch.as_tensor(u0, dtype=torch.float32)
    r0 = None if rho0 is None else slabs.slab_of(torch.as_tensor(rho0, dtype=torch.float32).cuda(), D.plan, *dims[:2])
    D.L.init(r0, slabs.slab_of(u0t.cuda().reshape(3, -1), D.plan, *dims[:2]))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, kms, launches = time_steps(D.L, args.steps, args.warmup, torch)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    D.L.close()
    ms_max, _ = job_throughput(ms, 1, 1, dist, torch)
    if rank != 0:
        return
    nloc = dims[0] * dims[1] * D.plan.nz_local
    line = {
        "metric": "MLUPS", "value": N * args.steps / (ms_max * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "D3Q19 FP32 %d^3 periodic Taylor-Green, u0 0.02, rotated Theta, tau 0.6, shifted "
                               "FP32 storage, cut into %d z-slabs" % (n, world),
                   "cells": N, "parallelism": "z-slabs, halo planes over torch.distributed after every step",
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": 152 * nloc / (kms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 152 * nloc / (kms * 1e-3) / 1e9 / peak, "traffic": None, "peak_source": peak_src,
                     "kernel": "k_step_pull<19, FP32_SHIFTED> (slab objects) + halo exchange, rank 0",
                     "note": "per-step event time includes the halo pack, exchange and unpack"},
        "cpu_baseline": None, "e2e": None, "clocks": clk.summary(), "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_profile(args, torch, lbm):
    """Small case for ncu: --kernel fwd runs warmup + steps forward launches; --kernel adjoint
    runs one short adjoint (seed, recompute, adjoint steps)."""
    kind = ("ade_porous" if args.ade else "porous") if args.porous else "ade" if args.ade else "tg"
    L, _ = make_ctx(args.lattice, args.n, args.storage, args.scheme, kind, torch, lbm, use_graphs=-1)
    if args.kernel == "fwd":
        L.step(args.warmup + args.steps)
    else:
        L.step(args.steps)
        g = torch.randn(L.d, L.N, device="cuda", dtype=torch.float64 if args.storage == "fp64" else torch.float32)
        L.adjoint(g, args.steps, max(1, args.steps // 2))
    torch.cuda.synchronize()
    print(json.dumps({"profile": True, "lattice": args.lattice, "n": args.n, "storage": args.storage,
                      "scheme": args.scheme, "kernel": args.kernel, "launches": L.launches}))
    L.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="bench", choices=["bench", "sweep", "profile", "slabs", "oracle"])
    ap.add_argument("--no-extras", action="store_true", help="contract line without sub-measurements/e2e/cpu")
    ap.add_argument("--only", default="", help="sweep: substring filter on case names")
    ap.add_argument("--lattice", type=int, default=19)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--storage", default="fp32s")
    ap.add_argument("--scheme", default="pull")
    ap.add_argument("--kernel", default="fwd", choices=["fwd", "adjoint"])
    ap.add_argument("--porous", action="store_true")
    ap.add_argument("--ade", action="store_true", help="profile: the scalar advection-diffusion workload")
    ap.add_argument("--sharded", action="store_true",
                    help="one box cut into z-slabs over the ranks (strong scaling) instead of replicas")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "oracle":  # the oracle on a bounded sample of each workload (host cores only)
        import oracle
        for cfg, v, sample in oracle_per_config():
            print(json.dumps({"oracle": True, "config": cfg, "value": v, "unit": "MLUPS", "cores": oracle.threads(),
                              "kind": "oracle", "sample": sample}), flush=True)
        return

    import torch
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.mode == "sweep":
        run_sweep(args, torch, lbm)
        return
    if args.mode == "profile":
        run_profile(args, torch, lbm)
        return
    if args.mode == "slabs":
        run_slabs(args, torch, lbm)
        return

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.sharded:
        run_sharded(args, torch, lbm, dist, world, rank, local)
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_src = measured_peak()
    q, n, storage = 19, 256, "fp32s"
    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_extras) else None

    # timed region: K forward steps of the 256^3 D3Q19 FP32 workload (independent replica per rank)
    L, nf = make_ctx(q, n, storage, "pull", "tg", torch, lbm)
    N = L.N
    barrier()
    with ClockSampler(local) as clk:
        ms, kms, launches = time_steps(L, args.steps, args.warmup, torch)
    barrier()
    L.close()
    del L
    ms, mlups = job_throughput(ms, N, args.steps, dist, torch, device="cuda")
    bpc = 2 * q * ELEM[storage]
    achieved = bpc * N / (kms * 1e-3) / 1e9
    rec = NCU_TRAFFIC.get("d3q19_fp32s_pull")
    fresh = bool(rec) and rec.get("traffic_bytes") is not None and rec.get("kernel_sha") == kernel_source_hash()
    traffic = rec["traffic_bytes"] if fresh else None
    traffic_note = ("ncu capture of the same kernel source (sha %s)" % rec["kernel_sha"] if fresh else
                    "null: no ncu capture of the current kernel source (sha %s)" % kernel_source_hash())
    torch.cuda.empty_cache()

    sub, e2e = {}, None
    if not args.no_extras:
        if rank == 0:
            r16 = variant(19, 256, "fp16s", "pull", "tg", max(10, args.steps // 2), args.warmup, torch, lbm, peak)
            sub["fwd_fp16s_256"] = {k: r16[k] for k in ("mlups_all", "kernel_gbs", "frac", "kernel_ms")}
            msa, Na, la, msa1, _ = time_adjoint(19, 128, "fp32s", "pull", 200, 20, torch, lbm)
            sub["adjoint_fp32s_128"] = {"mlups": Na * 200 / (msa * 1e-3) / 1e6, "steps": 200, "checkpoint_every": 20,
                                       "launches": la, "mlups_first_call": Na * 200 / (msa1 * 1e-3) / 1e6,
                                       "note": "wall time of lbm_adjoint incl. forward recompute (second call "
                                               "on the same forward run; the first also allocates its buffers)"}
        msE, h2d, d2h = time_e2e(q, n, storage, args.steps, torch, lbm)
        e2e = {"value": N * args.steps * world / (msE * 1e-3) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "per job: one pinned upload of (rho0, u0), init, K = %d steps, moments, one download "
                       "of u; bytes amortised over the K steps" % args.steps}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "D3Q19 FP32 256^3 periodic Taylor-Green, u0 0.02, rotated Theta "
                               "R diag(0.36,0.33,0.30) R^T, tau 0.6; populations stored as FP32 f - r_i "
                               "(the library's default storage), FP32 arithmetic",
                   "cells": N, "l2": "inputs larger than L2 (2 x %.2f GB populations)" % (q * N * 4 / 1e9),
                   "parallelism": "independent replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_note, "peak_source": peak_src,
                     "kernel": "k_step_pull<19, FP32_SHIFTED>",
                     "bytes_per_cell": bpc, "kernel_ms_mean": kms},
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

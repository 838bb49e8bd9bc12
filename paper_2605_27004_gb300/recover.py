"""Recovery of an anisotropy tensor from a target flow field with the discrete adjoint.

Workload (D3Q19, periodic n^3, FP32 storage, FP64 gradient accumulation): the initial velocity
is a seeded solenoidal field of random Fourier modes (|k| <= 4, max |u| = 0.02); the target is
u*(T) produced with a hidden SPD Theta* (eigenvalues in [0.29, 0.38]); starting from
Theta = c_s^2 I, Adam minimises L = mean over cells of |u(T) - u*|^2, with dL/dTheta from
``lbm_adjoint`` (checkpoints every K steps recorded during each forward run).

    python -m paper_2605_27004_gb300.recover --n 128 --steps 2000 --K 100 --iters 50
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import inputs
from . import lbm as _lbm
from .autograd import simulate, theta_matrix, theta_vector

CS2 = 1.0 / 3.0


def recover_theta(n=128, steps=2000, K=100, iters=50, lr=4e-3, tau=0.6, storage="fp32s", seed=inputs.SEED_BASE + 4,
                  log=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    theta_true = theta_vector(inputs.theta_spd(seed + 10))
    _, u0 = inputs.random_fourier_modes(n, 4.0, 0.02, seed)
    dt = torch.float64 if storage == "fp64" else torch.float32
    u0_t = torch.as_tensor(u0, dtype=dt, device=dev)
    sim = _lbm.LBM(19, n, n, n, tau, theta_matrix(theta_true, 3), storage=storage)
    with torch.no_grad():
        target = simulate(u0_t, torch.as_tensor(theta_true), tau, sim, steps, K).clone()
    theta = torch.tensor(theta_vector(CS2 * np.eye(3)), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    hist = []
    t0 = time.perf_counter()
    for it in range(iters):
        u = simulate(u0_t, theta, tau, sim, steps, K)
        loss = ((u - target) ** 2).sum(dim=0).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        err = float(np.linalg.norm(theta_matrix(theta.detach().numpy(), 3) - theta_matrix(theta_true, 3)) /
                    np.linalg.norm(theta_matrix(theta_true, 3)))
        rec = {"iter": it, "loss": float(loss.detach()), "rel_err_theta": err}
        hist.append(rec)
        if log:
            log(rec)
    wall = time.perf_counter() - t0
    sim.close()
    return {"theta": theta.detach().numpy().tolist(), "theta_true": theta_true.tolist(), "history": hist,
            "wall_s": wall, "n": n, "steps": steps, "K": K, "iters": iters}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--K", type=int, default=100)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--lr", type=float, default=4e-3)
    ap.add_argument("--storage", default="fp32s")
    args = ap.parse_args()
    out = recover_theta(args.n, args.steps, args.K, args.iters, args.lr, storage=args.storage,
                        log=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps({k: v for k, v in out.items() if k != "history"}))


if __name__ == "__main__":
    main()

"""Shared helpers of the GPU parity tests: run the library and the oracle on the same inputs."""
import numpy as np

import oracle
from paper_2605_27004_gb300 import inputs

CS2 = 1.0 / 3.0


def perm_lib_to_oracle(q):
    """perm[i] = oracle direction index of the library's direction i (matched by velocity)."""
    from paper_2605_27004_gb300 import lbm
    cl, _ = lbm.lattice_info(q)
    co, _, _ = oracle.lattice(q)
    look = {tuple(v): j for j, v in enumerate(co)}
    return np.array([look[tuple(v)] for v in cl])


def rand_theta(seed, d, spread=0.04):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    return CS2 * np.eye(d) + spread * (A + A.T) / 2


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_run(q, dims, tau, Theta, rho0, u0, steps, solid=None, order=3, storage="fp64", scheme="pull", **kw):
    """storage=None runs the library's default storage form."""
    import torch
    from paper_2605_27004_gb300 import lbm
    nx, ny, nz = dims
    if storage is not None:
        kw["storage"] = storage
    L = lbm.LBM(q, nx, ny, nz, tau, Theta, solid=solid, scheme=scheme, order=order, **kw)
    L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    L.step(steps)
    rho, u, Pi = L.moments(Pi=True)
    f = L.populations()
    torch.cuda.synchronize()
    out = dict(rho=rho.double().cpu().numpy(), u=u.double().cpu().numpy(), Pi=Pi.double().cpu().numpy(),
               f=f.double().cpu().numpy(), ctx=L)
    return out


def oracle_run(q, dims, tau, Theta, rho0, u0, steps, solid=None, order=3):
    pb = oracle.Problem(q, *dims, tau, Theta, solid=solid, order=order)
    f, rho, u, Pi = pb.simulate(rho0, u0, steps)
    return dict(f=f, rho=rho, u=u, Pi=Pi, pb=pb)

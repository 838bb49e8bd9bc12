"""PyTorch autograd wrapper around the library's forward run and discrete adjoint.

``LBMFunction.apply(u0, theta, tau, sim, n, K)`` returns u(n) of the lattice run started from
f(0) = feq(rho0, u0; Theta) (Sec. 4 initialises from the macroscopic fields); its backward calls
``lbm_adjoint`` and returns dL/du0, dL/dtheta and dL/dtau. ``theta`` holds the independent
entries of the symmetric anisotropy tensor Theta = c_s^2 A^{-1} (Eq. K-term): (xx, yy, xy) in 2D,
(xx, yy, zz, xy, xz, yz) in 3D, so an off-diagonal entry moves Theta_ab and Theta_ba together and
its gradient is dL/dTheta_ab + dL/dTheta_ba, which is what the library reports.

The forward records checkpoints every K steps while it runs (``lbm_record_checkpoints``), so the
backward recomputes only inside segments. All arithmetic runs in the library's kernels; this
module only moves tensors and scalars across the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm as _lbm

_IDX2 = [(0, 0), (1, 1), (0, 1)]
_IDX3 = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def theta_matrix(theta, d: int) -> np.ndarray:
    """Symmetric d x d Theta from its independent entries (xx, yy, [zz,] xy, [xz, yz])."""
    t = np.asarray(theta, dtype=np.float64).reshape(-1)
    M = np.zeros((d, d))
    for k, (a, b) in enumerate(_IDX2 if d == 2 else _IDX3):
        M[a, b] = M[b, a] = t[k]
    return M


def theta_vector(Theta) -> np.ndarray:
    Theta = np.asarray(Theta, dtype=np.float64)
    d = Theta.shape[0]
    return np.array([Theta[a, b] for a, b in (_IDX2 if d == 2 else _IDX3)])


class LBMFunction(torch.autograd.Function):
    """u(n) = LBM^n(feq(rho0, u0; theta)); differentiable in u0, theta and tau."""

    @staticmethod
    def forward(ctx, u0, theta, tau, sim: "_lbm.LBM", n: int, K: int, rho0=None):
        sim.set_params(float(tau), theta_matrix(theta.detach().cpu().numpy(), sim.d))
        sim.record_checkpoints(int(K))
        sim.init(rho0, u0.detach())
        sim.step(int(n))
        _, u, _ = sim.moments(rho=False, u=True)
        ctx.sim, ctx.n, ctx.K = sim, int(n), int(K)
        ctx.theta_dtype, ctx.tau_is_tensor = theta.dtype, isinstance(tau, torch.Tensor)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        sim = ctx.sim
        sim.adjoint(grad_u.contiguous(), ctx.n, ctx.K)
        dth, dtau, du0 = sim.gradients(du0=ctx.needs_input_grad[0])
        g_theta = torch.as_tensor(dth, dtype=ctx.theta_dtype)
        g_tau = torch.tensor(dtau, dtype=torch.float64) if ctx.tau_is_tensor else None
        return du0, g_theta, g_tau, None, None, None, None


def simulate(u0, theta, tau, sim, n, K=0, rho0=None):
    """Differentiable forward run: see :class:`LBMFunction`."""
    return LBMFunction.apply(u0, theta, tau, sim, n, K, rho0)

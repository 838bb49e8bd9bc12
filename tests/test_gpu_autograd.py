"""torch.autograd wrapper, finite differences of the GPU forward run, and Theta recovery.

The paper has no adjoint; the references are central finite differences of the library's own
FP64 forward run (independent of the adjoint kernels) and the recovery of a hidden Theta*.
"""
import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


def test_gradients_match_finite_differences_fp64():
    """L = sum g.u(n) on a 20x18x16 D3Q19 box with walls, FP64 storage: adjoint dL/dTheta (6),
    dL/dtau and dL/du0 (random direction) against central differences (h = 1e-6) of the
    library's forward run."""
    import torch
    from paper_2605_27004_gb300 import lbm
    from paper_2605_27004_gb300.autograd import simulate, theta_matrix, theta_vector
    dims, n, K, tau = (20, 18, 16), 30, 7, 0.65
    N = int(np.prod(dims))
    solid = inputs.channel_walls(*dims)
    rho0, u0 = inputs.noise_field(N, 3, 0.03, 3, rho_amp=0.01)
    u0 *= (1 - solid)[None, :]
    rng = np.random.default_rng(4)
    g = torch.as_tensor(rng.standard_normal((3, N)) * (1 - solid)[None, :], device="cuda")
    th0 = theta_vector(inputs.theta_rotated([0.36, 0.33, 0.30], 5))
    sim = lbm.LBM(19, *dims, tau, theta_matrix(th0, 3), solid=solid, storage="fp64")
    u0t = torch.as_tensor(u0, device="cuda").requires_grad_(True)
    theta = torch.tensor(th0, requires_grad=True)
    taut = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
    L = (simulate(u0t, theta, taut, sim, n, K) * g).sum()
    L.backward()

    def loss(th, ta, uu):
        with torch.no_grad():
            return float((simulate(torch.as_tensor(uu, device="cuda"), torch.as_tensor(th), ta, sim, n, K) * g).sum())

    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (loss(th0 + e, tau, u0) - loss(th0 - e, tau, u0)) / (2 * h)
        assert abs(theta.grad[k].item() - fd) <= 1e-6 * max(1.0, abs(fd)), (k, theta.grad[k].item(), fd)
    fd = (loss(th0, tau + h, u0) - loss(th0, tau - h, u0)) / (2 * h)
    assert abs(taut.grad.item() - fd) <= 1e-6 * max(1.0, abs(fd))
    v = rng.standard_normal((3, N)) * (1 - solid)[None, :]
    fd = (loss(th0, tau, u0 + h * v) - loss(th0, tau, u0 - h * v)) / (2 * h)
    got = float((u0t.grad.cpu().numpy() * v).sum())
    assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd))


def test_theta_recovery_small():
    """Adam on Theta from c_s^2 I recovers a hidden SPD Theta* (32^3, 300 steps, K = 30)."""
    from paper_2605_27004_gb300.recover import recover_theta
    out = recover_theta(n=32, steps=300, K=30, iters=40, lr=4e-3)
    h = out["history"]
    assert h[-1]["loss"] < 1e-2 * h[0]["loss"]
    assert h[-1]["rel_err_theta"] < 0.2 * h[0]["rel_err_theta"]

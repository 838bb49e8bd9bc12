"""FP16 storage shifted by the rest equilibrium r_i = feq_i(rho0, 0; Theta) (the library's
LBM_FP16_SHIFTED) against the shift by the lattice weights alone, f_i - w_i rho0
(LBM_FP16_WSHIFTED), with the same FP32 arithmetic.

When Theta != cs2 I the rest equilibrium differs from w_i rho0 by 9/2 w_i rho0 h_i with
h_i = c_i.K~.c_i - cs2 tr K~ (Eq. 3rd_order_equilibrium at u = 0), so the weight-shifted form
stores that offset on top of the O(u) deviation and rounds it to 11 bits. At Theta = cs2 I the
two shifts coincide (h_i = 0) and so do the runs. The full-size comparison at the porous
workload's Theta = diag(0.38, 0.33, 0.29) is in test_gpu_porous_512.py."""
import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(q, dims, Th, storage, rho0, u0, steps, tau, solid=None):
    import torch
    from paper_2605_27004_gb300 import lbm
    L = lbm.LBM(q, *dims, tau, Th, solid=solid, storage=storage)
    dt = L.dtype
    L.init(None if rho0 is None else torch.as_tensor(rho0, dtype=dt), torch.as_tensor(u0, dtype=dt))
    m0, _ = L.totals()
    L.step(steps)
    m1, _ = L.totals()
    u = L.moments(rho=False)[1].double()
    f = L.populations()
    L.close()
    return u, f, (m1 - m0) / m0


def test_shifts_coincide_for_isotropic_theta():
    """Theta = cs2 I: r_i = w_i rho0 exactly, so both FP16 forms store the same numbers; with an odd
    nx both run the one-cell kernels and agree bit for bit."""
    import torch
    q, dims = 19, (33, 12, 10)
    N = int(np.prod(dims))
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 90, rho_amp=0.02)
    Th = np.eye(3) / 3
    _, fs, _ = _run(q, dims, Th, "fp16s", rho0, u0, 25, 0.7)
    _, fw, _ = _run(q, dims, Th, "fp16w", rho0, u0, 25, 0.7)
    assert torch.equal(fs, fw)


def test_weight_shift_costs_accuracy_at_the_taylor_green_theta():
    """The 256^3 Taylor-Green workload (rotated Theta = R diag(0.36, 0.33, 0.30) R^T, u0 = 0.02,
    tau 0.6), 1000 steps: both FP16 forms against the FP64 mode (which matches the oracle to
    1e-13). The r_i-shifted form meets the 1e-3 bar; the weight-shifted one is less accurate."""
    import torch
    n, steps = 256, 1000
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, uu = inputs.taylor_green_3d(n, 0.02)
    ref, _, _ = _run(19, (n, n, n), Th, "fp64", rho0, uu, steps, 0.6)
    err, drift = {}, {}
    for storage in ("fp16s", "fp16w"):
        u, _, dm = _run(19, (n, n, n), Th, storage, rho0, uu, steps, 0.6)
        err[storage] = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
        drift[storage] = dm
        print(f"{storage}: relative u L2 {err[storage]:.3e}, mass drift {dm:.2e}")
        torch.cuda.empty_cache()
    assert err["fp16s"] < 1e-3
    assert err["fp16w"] > err["fp16s"]

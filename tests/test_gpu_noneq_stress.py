"""Non-equilibrium second moment against the Chapman-Enskog perturbation moment (App. G):
M_ab(f1) = -tau rho (Theta_bc d_c u_a + Theta_ac d_c u_b) in lattice units (c_s^2 A^{-1} = Theta)
for the third-order equilibrium. With the second-order equilibrium the third moment lacks the K
terms (Eq. mom_diff2), and for a solenoidal field the same derivation gives the isotropic
-tau rho c_s^2 (d_b u_a + d_a u_b) (App. G closing remark). The pre-collision Pi from
lbm_moments minus the equilibrium part rho (Theta + u u) is compared with both on a
small-amplitude shear wave, where the gradients are known in closed form."""
import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


# D3Q27 only: D3Q19 does not reproduce the third equilibrium moment the derivation uses (it has
# no corner velocities), and measures 8 % off the anisotropic formula here (a lattice limit).
@pytest.mark.parametrize("q,order", [(27, 3), (27, 2)])
def test_nonequilibrium_stress_matches_chapman_enskog(q, order):
    import torch
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    n, tau, amp = 64, 0.8, 1e-4
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    # transverse wave along y, velocity along x, small enough to be linear
    rho0, u0 = inputs.shear_wave(n, n, 8, k_axis=1, u_axis=0, amp=amp)
    L = lbm.LBM(q, n, n, 8, tau, Th, storage="fp64", order=order)
    L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    L.step(300)  # let the initial non-equilibrium transient relax
    rho, u, Pi = (t.cpu().numpy() for t in L.moments(Pi=True))
    N = n * n * 8
    _, y, _ = inputs._grid(n, n, 8)
    k = 2 * np.pi / n
    # u_x = a(t) sin(k y): fit a(t) and use the exact derivative d_y u_x = a k cos(k y)
    s, c = np.sin(k * y), np.cos(k * y)
    a = (u[0] * s).sum() / (s * s).sum()
    grad = np.zeros((3, 3, N))  # grad[a, c] = d_c u_a
    grad[0, 1] = a * k * c
    def predicted(T):
        ce = np.zeros((6, N))
        for p, (al, be) in enumerate(PAIRS):
            ce[p] = -tau * rho * (np.einsum("c,cn->n", T[be], grad[al]) + np.einsum("c,cn->n", T[al], grad[be]))
        return ce

    neq = np.zeros((6, N))
    for p, (al, be) in enumerate(PAIRS):
        neq[p] = Pi[p] - rho * (Th[al, be] + u[al] * u[be])
    aniso, iso = predicted(Th), predicted(np.eye(3) / 3)
    right, wrong = (aniso, iso) if order == 3 else (iso, aniso)
    err = np.linalg.norm(neq - right) / np.linalg.norm(right)
    err_other = np.linalg.norm(neq - wrong) / np.linalg.norm(wrong)
    print(q, order, "rel err", err, "other", err_other)
    assert err < 0.03
    assert err_other > 3 * err

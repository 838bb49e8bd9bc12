"""Parity at the full workload sizes, in the launch configuration the benchmark times.

The oracle cannot run these boxes, so sampled outputs are checked one by one: after k steps the
library's pre-collision populations f(t) and f(t+1) are fetched (lbm_populations), and for a
seeded sample of fluid cells x every f_i(x, t+1) is recomputed from the oracle's one-cell BGK
collision of the source cell: f_i(x, t+1) = f*_i(x - c_i) if x - c_i is fluid, else
f*_opp(i)(x) (half-way bounce-back). Tolerances: FP32 arithmetic on O(1) populations, 2e-6
absolute; FP16 storage rounds f - r to 11 bits, 2e-4 absolute (|f - r| < 0.2).
"""
import numpy as np
import pytest

import oracle
from paper_2605_27004_gb300 import inputs

from gpu_util import perm_lib_to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


def _check_samples(L, q, dims, Th, tau, solid, steps, nsamp, tol, seed):
    import torch
    from paper_2605_27004_gb300 import lbm
    nx, ny, nz = dims
    N = nx * ny * nz
    L.step(steps)
    fa = L.populations()
    L.step(1)
    fb = L.populations()
    c, _ = lbm.lattice_info(q)
    co, _, _ = oracle.lattice(q)
    perm = perm_lib_to_oracle(q)           # library direction -> oracle direction
    inv = np.argsort(perm)                  # oracle direction -> library direction
    opp = np.array([0] + [i + 1 if i % 2 else i - 1 for i in range(1, q)])
    rng = np.random.default_rng(seed)
    cand = rng.integers(0, N, size=4 * nsamp)
    if solid is not None:
        cand = cand[solid[cand] == 0]
    xs = cand[:nsamp]

    def coords(n):
        return n % nx, (n // nx) % ny, n // (nx * ny)

    def index(x, y, z):
        return (x % nx) + nx * ((y % ny) + ny * (z % nz))

    # every source cell needed: the samples and their neighbours x - c_i
    need = set()
    for n in xs:
        x, y, z = coords(int(n))
        need.add(int(n))
        for i in range(q):
            need.add(int(index(x - c[i, 0], y - c[i, 1], z - c[i, 2])))
    need = np.array(sorted(need))
    fa_s = fa[:, torch.as_tensor(need, device=fa.device)].double().cpu().numpy()  # [q, len(need)]
    fb_s = fb[:, torch.as_tensor(xs, device=fb.device)].double().cpu().numpy()
    col = {}
    for k, n in enumerate(need):
        if solid is not None and solid[n]:
            continue
        f_or = fa_s[:, k][inv]  # library order -> oracle order
        col[int(n)] = oracle.collide_cell(q, f_or, tau, Th)[perm]  # back to library order
    worst = 0.0
    for k, n in enumerate(xs):
        x, y, z = coords(int(n))
        for i in range(q):
            s = int(index(x - c[i, 0], y - c[i, 1], z - c[i, 2]))
            if solid is not None and solid[s]:
                expect = col[int(n)][opp[i]]
            else:
                expect = col[s][i]
            worst = max(worst, abs(fb_s[i, k] - expect))
    print("max |f_gpu - f_oracle| over samples:", worst)
    assert worst < tol


def test_bench_workload_d3q19_fp32_256():
    """The benchmark's workload and launch path: D3Q19 FP32 256^3 Taylor-Green, rotated Theta,
    tau 0.6, one-cell pull kernel with the FP32 momentum identity."""
    import torch
    from paper_2605_27004_gb300 import lbm
    n = 256
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    L = lbm.LBM(19, n, n, n, 0.6, Th, storage="fp32")
    L.init(torch.as_tensor(rho0, dtype=torch.float32), torch.as_tensor(u0, dtype=torch.float32))
    _check_samples(L, 19, (n, n, n), Th, 0.6, None, 20, 600, 2e-6, 1)


def test_porous_d3q27_512_fp32_and_fp16():
    """The porous workload at full size: D3Q27 512^3, overlapping spheres, walls at z = 0, 511,
    u_x = 0.03 in the fluid, tau 0.7, Theta = diag(0.38, 0.33, 0.29); FP32 and FP16-shifted."""
    import torch
    from paper_2605_27004_gb300 import lbm
    n = 512
    solid = inputs.porous_spheres(n, n, n, seed=inputs.SEED_BASE + 3)
    N = n ** 3
    u0 = np.zeros((3, N), dtype=np.float32)
    u0[0] = 0.03 * (1 - solid)
    Th = np.diag([0.38, 0.33, 0.29])
    for storage, tol in (("fp32", 2e-6), ("fp16s", 2e-4)):
        L = lbm.LBM(27, n, n, n, 0.7, Th, solid=solid, storage=storage)
        L.init(None, torch.as_tensor(u0))
        _check_samples(L, 27, (n, n, n), Th, 0.7, solid, 10, 400, tol, 2)
        L.close()
        torch.cuda.empty_cache()


def test_aa_d3q19_768_fp16():
    """The largest Taylor-Green box: D3Q19 768^3 Taylor-Green, FP16-shifted, AA in place
    (samples after an odd and after an even number of steps)."""
    import torch
    from paper_2605_27004_gb300 import lbm
    n = 768
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    k = 2 * np.pi / n
    ax = torch.arange(n, device="cuda", dtype=torch.float32) * k
    s_, c_ = torch.sin(ax), torch.cos(ax)
    u0 = torch.zeros((3, n, n, n), device="cuda", dtype=torch.float32)
    u0[0] = 0.02 * s_[None, None, :] * c_[None, :, None] * c_[:, None, None]
    u0[1] = -0.02 * c_[None, None, :] * s_[None, :, None] * c_[:, None, None]
    L = lbm.LBM(19, n, n, n, 0.6, Th, storage="fp16s", scheme="aa")
    L.init(None, u0.reshape(3, -1))
    del u0
    _check_samples(L, 19, (n, n, n), Th, 0.6, None, 5, 300, 2e-4, 3)
    _check_samples(L, 19, (n, n, n), Th, 0.6, None, 0, 300, 2e-4, 4)

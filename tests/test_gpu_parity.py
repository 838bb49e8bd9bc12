"""GPU parity: the CUDA library against the FP64 oracle on identical seeded inputs.

Every test runs the library through its C ABI (ctypes binding) on cuda:0 and compares element
by element with the oracle. Sizes span several thread blocks with ragged tails in x and y.
Tolerances: FP64 storage 1e-12 relative (populations to 1e-13 absolute, values <= 0.5);
FP32-shifted 1e-5 and FP16-shifted 1e-3 relative velocity L2 after 1000 steps.
"""
import numpy as np
import pytest

import oracle
from paper_2605_27004_gb300 import inputs

from gpu_util import gpu_run, oracle_run, perm_lib_to_oracle, rand_theta, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


GEOMS = {9: (70, 37, 1), 19: (45, 13, 9), 27: (37, 11, 10)}


def _mask(q, dims, kind, seed=5):
    N = int(np.prod(dims))
    if kind is None:
        return None
    if kind == "random":
        return inputs.random_mask(N, 0.2, seed)
    if kind == "walls":
        nx, ny, nz = dims
        if q == 9:
            m = np.zeros((ny, nx), np.uint8)
            m[0] = 1
            m[-1] = 1
            return m.reshape(-1)
        return inputs.channel_walls(nx, ny, nz)
    raise ValueError(kind)


@pytest.mark.parametrize("q", [9, 19, 27])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("mask", [None, "random", "walls"])
@pytest.mark.parametrize("order,steps", [(3, 41), (2, 40)])
def test_fp64_populations_match_oracle(q, scheme, mask, order, steps):
    dims = GEOMS[q]
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    Th = rand_theta(10 + q, d)
    solid = _mask(q, dims, mask)
    rho0, u0 = inputs.noise_field(N, d, 0.05, 20 + q, rho_amp=0.02)
    g = gpu_run(q, dims, 0.7, Th, rho0, u0, steps, solid=solid, order=order, storage="fp64", scheme=scheme)
    o = oracle_run(q, dims, 0.7, Th, rho0, u0, steps, solid=solid, order=order)
    perm = perm_lib_to_oracle(q)
    f_or = o["f"][:, perm].T
    assert np.abs(g["f"] - f_or).max() < 1e-13
    fl = slice(None) if solid is None else (solid == 0)
    assert np.abs(g["rho"] - o["rho"]).max() < 1e-13
    assert rel_l2(g["u"][:, fl], o["u"][:, fl]) < 1e-12
    assert np.abs(g["Pi"] - o["Pi"]).max() < 1e-13
    if solid is not None:
        assert np.all(g["rho"][solid == 1] == 0)


def test_shear_wave_d2q9_64_fp64():
    """D2Q9, FP64, 64x64 periodic, tau 0.8, Theta [[0.36,0.02],[0.02,0.30]], u_x = 0.01 sin(2 pi y/64)
    + 1e-4 noise, 1000 steps: fields, totals and the shear-wave decay rate."""
    q, dims, tau = 9, (64, 64, 1), 0.8
    Th = np.array([[0.36, 0.02], [0.02, 0.30]])
    rho0, u0 = inputs.shear_wave_2d(64, 64, 0.01, 1e-4, seed=inputs.SEED_BASE + 1)
    g = gpu_run(q, dims, tau, Th, rho0, u0, 1000, storage="fp64")
    o = oracle_run(q, dims, tau, Th, rho0, u0, 1000)
    assert rel_l2(g["u"], o["u"]) < 1e-12
    assert rel_l2(g["rho"], o["rho"]) < 1e-12
    m_g, p_g = g["ctx"].totals()
    m_o, p_o = o["pb"].totals(o["f"])
    assert abs(m_g - m_o) < 1e-12 * m_o
    assert np.abs(p_g - p_o).max() < 1e-12 * m_o
    # decay of the sin(2 pi y / 64) projection against the exact linear rate
    from oracle import linear
    _, y, _ = inputs._grid(64, 64, 1)
    s = np.sin(2 * np.pi * y / 64)
    a0 = (u0[0] * s).sum()
    a1 = (g["u"][0] * s).sum()
    rate = -np.log(a1 / a0) / 1000
    lin = linear.shear_rate(9, Th, tau, [0, 2 * np.pi / 64], [1, 0])
    assert abs(rate - lin) / lin < 5e-3


@pytest.mark.parametrize("n,storage,tol", [(32, "default", 1e-5), (32, "fp32s", 1e-5), (32, "fp16s", 1e-3),
                                           (64, "default", 1e-5), (64, "fp32s", 1e-5), (64, "fp16s", 1e-3),
                                           (32, "fp32", 1e-4), (64, "fp32", 1e-5)])
def test_reduced_precision_taylor_green_d3q19(n, storage, tol):
    """D3Q19 Taylor-Green (u0 = 0.02, rotated Theta, tau 0.6; the 256^3 workload's recipe at n^3),
    1000 steps, against the FP64 oracle. The default storage (shifted FP32) meets 1e-5 relative
    velocity L2. At 32^3 the vortex decays to 2 % of its amplitude, the hardest case for relative
    accuracy; the non-default plain FP32 storage, which rounds f ~ w_i instead of f - r_i, then
    reaches ~4e-5 and is held to its own documented bound of 1e-4 there."""
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    rho0, u0 = inputs.taylor_green_3d(n, 0.02)
    g = gpu_run(19, (n, n, n), 0.6, Th, rho0, u0, 1000, storage=None if storage == "default" else storage)
    o = oracle_run(19, (n, n, n), 0.6, Th, rho0, u0, 1000)
    err = rel_l2(g["u"], o["u"])
    print(f"{storage}: rel u L2 = {err:.3e}")
    assert err < tol


@pytest.mark.parametrize("storage,tol", [("fp32s", 1e-5), ("fp16s", 1e-3)])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_reduced_precision_porous_d3q27(storage, tol, scheme):
    """D3Q27 porous medium between walls (the 512^3 porous recipe at 40x36x30), u_x = 0.03, 300 steps."""
    dims = (40, 36, 30)
    solid = inputs.porous_spheres(*dims, rmin=3, rmax=6, seed=inputs.SEED_BASE + 3)
    N = int(np.prod(dims))
    u0 = np.zeros((3, N))
    u0[0] = 0.03 * (1 - solid)
    rho0 = np.ones(N)
    Th = np.diag([0.38, 0.33, 0.29])
    g = gpu_run(27, dims, 0.7, Th, rho0, u0, 300, solid=solid, storage=storage, scheme=scheme)
    o = oracle_run(27, dims, 0.7, Th, rho0, u0, 300, solid=solid)
    fl = solid == 0
    err = rel_l2(g["u"][:, fl], o["u"][:, fl])
    print(f"{storage}/{scheme}: rel u L2 = {err:.3e}")
    assert err < tol
    m_g, _ = g["ctx"].totals()
    m_o, _ = o["pb"].totals(o["f"])
    assert abs(m_g - m_o) / m_o < 10 * tol


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_graph_replay_is_bit_identical(scheme):
    q, dims = 19, (33, 17, 12)
    N = int(np.prod(dims))
    Th = rand_theta(3, 3)
    rho0, u0 = inputs.noise_field(N, 3, 0.03, 4)
    a = gpu_run(q, dims, 0.6, Th, rho0, u0, 37, storage="fp32", scheme=scheme, use_graphs=1)
    b = gpu_run(q, dims, 0.6, Th, rho0, u0, 37, storage="fp32", scheme=scheme, use_graphs=-1)
    assert np.array_equal(a["f"], b["f"])


@pytest.mark.parametrize("storage", ["fp32", "fp16s", "fp64"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_state_roundtrip_bit_exact(storage, scheme):
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims = 27, (29, 14, 11)
    N = int(np.prod(dims))
    Th = rand_theta(8, 3)
    solid = inputs.random_mask(N, 0.15, 9)
    rho0, u0 = inputs.noise_field(N, 3, 0.03, 10)
    A = lbm.LBM(q, *dims, 0.65, Th, solid=solid, storage=storage, scheme=scheme)
    A.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    A.step(13)
    st = A.get_state()
    A.step(20)
    fa = A.populations().cpu()
    B = lbm.LBM(q, *dims, 0.65, Th, solid=solid, storage=storage, scheme=scheme)
    B.set_state(st)
    assert B.steps == 13
    B.step(20)
    fb = B.populations().cpu()
    assert torch.equal(fa, fb)


def test_error_paths():
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims = 19, (16, 8, 8)
    N = int(np.prod(dims))
    L = lbm.LBM(q, *dims, 0.7, np.eye(3) / 3)
    with pytest.raises(lbm.LBMError) as e:
        L.step(1)
    assert e.value.status == -9
    rho0, u0 = inputs.noise_field(N, 3, 0.01, 1)
    L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    L.step(3)
    with pytest.raises(lbm.LBMError) as e:
        L.adjoint(torch.zeros(3, N), 5)
    assert e.value.status == -7
    bad = rho0.copy()
    bad[17] = np.nan
    L.init(torch.as_tensor(bad), torch.as_tensor(u0))
    with pytest.raises(lbm.LBMError) as e:
        L.totals()
    assert e.value.status == -6
    C = lbm.LBM(q, *dims, 0.7, np.eye(3) / 3, check_every=2)
    C.init(torch.as_tensor(bad), torch.as_tensor(u0))
    with pytest.raises(lbm.LBMError) as e:
        C.step(4)
    assert e.value.status == -6


# Geometries for the two- and four-cells-per-thread kernels (FP16 storage; even nx two cells,
# nx a multiple of 128 four cells): rows shorter than a warp, rows of one and several warps
# (nx = 64, 128, 256, 384: the x wrap crosses a warp or a block boundary), odd nx (one-cell
# fallback), ragged ny and nz = 1
PAIR_GEOMS = [(19, (2, 5, 4)), (19, (64, 3, 3)), (19, (130, 3, 2)), (19, (46, 13, 9)), (27, (38, 11, 10)),
              (9, (98, 21, 1)), (19, (45, 7, 6)), (19, (128, 7, 5)), (27, (256, 5, 3)), (9, (384, 9, 1)),
              (19, (256, 3, 4)), (27, (100, 6, 5))]


@pytest.mark.parametrize("q,dims", PAIR_GEOMS)
@pytest.mark.parametrize("storage", ["fp32s", "fp32", "fp16s", "fp16w"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("mask", [None, "random"])
def test_fp32_and_fp16_kernels_match_oracle(q, dims, storage, scheme, mask):
    """Reduced-precision kernels (two cells per thread for even nx, one otherwise) on grids with
    one active lane per warp, exactly one warp per row, a ragged last warp, and walls; 40 steps.
    The default shifted FP32 storage stays below 2e-6 relative after 40 steps, FP16 storage below
    1e-3; the non-default plain FP32 storage (f ~ 0.3 rounded to ~2e-8 absolute per step against
    u ~ 1e-3) is held to its documented 2e-5."""
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    Th = rand_theta(30 + q, d)
    solid = _mask(q, dims, mask, seed=31)
    rho0, u0 = inputs.noise_field(N, d, 0.05, 32 + q, rho_amp=0.02)
    g = gpu_run(q, dims, 0.7, Th, rho0, u0, 40, solid=solid, storage=storage, scheme=scheme)
    o = oracle_run(q, dims, 0.7, Th, rho0, u0, 40, solid=solid)
    fl = slice(None) if solid is None else (solid == 0)
    # fp16w (FP16 of f - w rho0, the comparison form for the r_i shift) rounds stored values that
    # carry r_i - w_i rho0 ~ 0.1 w_i at these Theta: measured 3.7e-3 after 40 steps
    tol = {"fp16s": 1e-3, "fp16w": 2e-2, "fp32": 2e-5, "fp32s": 2e-6}[storage]
    assert rel_l2(g["u"][:, fl], o["u"][:, fl]) < tol
    perm = perm_lib_to_oracle(q)
    f_or = o["f"][:, perm].T
    ftol = {"fp16s": 2e-3, "fp16w": 1e-2}.get(storage, 2e-6)
    assert np.abs(g["f"] - f_or).max() < ftol * np.abs(f_or).max()

"""GPU parity of the anisotropic advection-diffusion path (lbm_ade_create ...) against the
oracle's scalar scheme (oracle.ADEProblem) on identical seeded inputs.

FP64 storage: populations to 1e-13 times the largest population (41 steps; rounding order differs
between the pull gather and the oracle's push). Reduced precision: relative L2 of
phi - 1 (the transported variation) after 400 steps, FP32 forms 1e-5, FP16-shifted 1e-3, the
flow path's bars. Full size: sampled cells recomputed from the oracle's one-cell collision.
"""
import numpy as np
import pytest

import oracle
from paper_2605_27004_gb300 import inputs

from gpu_util import perm_lib_to_oracle, rand_theta, rel_l2

pytestmark = pytest.mark.gpu

GEOMS = {9: (70, 37, 1), 19: (45, 13, 9), 27: (37, 11, 10)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


def _mask(q, dims, kind):
    N = int(np.prod(dims))
    if kind is None:
        return None
    if kind == "random":
        return inputs.random_mask(N, 0.2, 7)
    nx, ny, nz = dims
    if q == 9:
        m = np.zeros((ny, nx), np.uint8)
        m[0] = 1
        m[-1] = 1
        return m.reshape(-1)
    return inputs.channel_walls(nx, ny, nz)


def _velocity(kind, d, N, seed):
    rng = np.random.default_rng(seed)
    if kind == "field":
        return 0.06 * rng.standard_normal((d, N))
    if kind == "const":
        return np.array([0.05, -0.03, 0.02])[:d]
    return None


def _oracle_u(u, d, N):
    if u is None:
        return np.zeros((d, N))
    u = np.asarray(u, dtype=np.float64)
    return np.tile(u[:, None], (1, N)) if u.size == d else u


def _gpu(q, dims, tau, Th, phi, u, steps, solid=None, order=3, storage="fp64", scheme="pull", **kw):
    import torch
    from paper_2605_27004_gb300 import lbm
    A = lbm.ADE(q, *dims, tau, Th, u=u, solid=solid, storage=storage, scheme=scheme, order=order, **kw)
    A.init(torch.as_tensor(phi))
    A.step(steps)
    out = {"phi": A.scalar().double().cpu().numpy(), "g": A.populations().double().cpu().numpy(), "ctx": A}
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("q", [9, 19, 27])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("mask", [None, "random", "walls"])
@pytest.mark.parametrize("vel,order", [("field", 3), ("const", 2), ("zero", 3)])
def test_fp64_scalar_populations_match_oracle(q, scheme, mask, vel, order):
    dims = GEOMS[q]
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    Th = rand_theta(30 + q, d)
    solid = _mask(q, dims, mask)
    rng = np.random.default_rng(50 + q)
    phi = 1.0 + 0.3 * rng.standard_normal(N)
    u = _velocity(vel, d, N, 60 + q)
    steps = 41
    g = _gpu(q, dims, 0.7, Th, phi, u, steps, solid=solid, order=order, scheme=scheme)
    P = oracle.ADEProblem(q, *dims, 0.7, Th, _oracle_u(u, d, N), solid=solid, order=order)
    go = P.init_scalar(phi)
    P.run_scalar(go, steps)
    perm = perm_lib_to_oracle(q)
    scale = max(1.0, np.abs(go).max())  # rest populations reach ~1 where phi ~ 2
    assert np.abs(g["g"] - go[:, perm].T).max() < 1e-13 * scale
    assert np.abs(g["phi"] - P.scalar(go)).max() < 1e-13 * max(1.0, np.abs(phi).max())
    if solid is not None:
        assert np.all(g["phi"][solid == 1] == 0)
    tot, flux = g["ctx"].totals()
    assert abs(tot - P.scalar(go).sum()) < 1e-12 * N


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-5), ("fp32s", 1e-5), ("fp16s", 1e-3)])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_reduced_precision_blob_in_taylor_green_d3q19(storage, tol, scheme):
    """A concentration blob carried by the Taylor-Green velocity field (frozen) with rotated Theta,
    48^3, tau 0.6, 400 steps."""
    n = 48
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    _, u = inputs.taylor_green_3d(n, 0.05)
    x, y, z = inputs._grid(n, n, n)
    phi = 1.0 + 0.5 * np.exp(-((x - 20.0) ** 2 + (y - 26.0) ** 2 + (z - 23.0) ** 2) / (2 * 5.0 ** 2))
    g = _gpu(19, (n, n, n), 0.6, Th, phi.astype(np.float32), u.astype(np.float32), 400, storage=storage,
             scheme=scheme)
    P = oracle.ADEProblem(19, n, n, n, 0.6, Th, u)
    go = P.init_scalar(phi)
    P.run_scalar(go, 400)
    ref = P.scalar(go)
    err = rel_l2(g["phi"] - 1.0, ref - 1.0)
    print(f"{storage}/{scheme}: rel (phi - 1) L2 = {err:.3e}")
    assert err < tol
    tot, _ = g["ctx"].totals()
    assert abs(tot - ref.sum()) < 10 * tol * np.abs(ref - 1).sum()


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-5), ("fp16s", 1e-3)])
def test_reduced_precision_porous_d3q27(storage, tol):
    """Scalar through the porous medium between walls (zero-flux), D3Q27, diagonal Theta."""
    dims = (40, 36, 30)
    solid = inputs.porous_spheres(*dims, rmin=3, rmax=6, seed=inputs.SEED_BASE + 3)
    N = int(np.prod(dims))
    u = np.zeros((3, N))
    u[0] = 0.03 * (1 - solid)
    rng = np.random.default_rng(77)
    phi = 1.0 + 0.4 * (rng.random(N) < 0.05)
    Th = np.diag([0.38, 0.33, 0.29])
    g = _gpu(27, dims, 0.7, Th, phi.astype(np.float32), u.astype(np.float32), 300, solid=solid, storage=storage)
    P = oracle.ADEProblem(27, *dims, 0.7, Th, u, solid=solid)
    go = P.init_scalar(phi)
    P.run_scalar(go, 300)
    ref = P.scalar(go)
    fl = solid == 0
    err = rel_l2(g["phi"][fl] - 1.0, ref[fl] - 1.0)
    print(f"{storage}: rel (phi - 1) L2 = {err:.3e}")
    assert err < tol


def test_velocity_changes_between_steps_fp64():
    """set_velocity between steps keeps the populations: 15 steps with u1, 16 with u2, then 10 with
    u = 0, against the oracle continuing the same g with each field."""
    q, dims = 19, (24, 10, 9)
    d, N = 3, int(np.prod(dims))
    Th = rand_theta(91, 3)
    rng = np.random.default_rng(92)
    phi = 1.0 + 0.2 * rng.random(N)
    u1 = 0.05 * rng.standard_normal((3, N))
    u2 = np.array([0.02, 0.04, -0.01])
    for scheme in ("pull", "aa"):
        import torch
        from paper_2605_27004_gb300 import lbm
        A = lbm.ADE(q, *dims, 0.8, Th, u=u1, storage="fp64", scheme=scheme)
        A.init(torch.as_tensor(phi))
        A.step(15)
        A.set_velocity(u2)
        A.step(16)
        A.set_velocity(None)
        A.step(10)
        ga = A.populations().cpu().numpy()
        go = oracle.ADEProblem(q, *dims, 0.8, Th, u1).init_scalar(phi)
        oracle.ADEProblem(q, *dims, 0.8, Th, u1).run_scalar(go, 15)
        oracle.ADEProblem(q, *dims, 0.8, Th, _oracle_u(u2, d, N)).run_scalar(go, 16)
        oracle.ADEProblem(q, *dims, 0.8, Th, np.zeros((d, N))).run_scalar(go, 10)
        assert np.abs(ga - go[:, perm_lib_to_oracle(q)].T).max() < 1e-13


def test_scalar_coupled_to_flow_through_the_velocity_view():
    """Zero-copy coupling: each step the flow's velocity u(t+1) is written by lbm_moments straight
    into the scalar context's velocity field, then the scalar steps (FP64, D2Q9, walls)."""
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims = 9, (40, 22, 1)
    N = int(np.prod(dims))
    Th = np.array([[0.36, 0.03], [0.03, 0.31]])
    ThS = np.array([[0.30, -0.04], [-0.04, 0.38]])
    solid = _mask(q, dims, "walls")
    rho0, u0 = inputs.noise_field(N, 2, 0.05, 93, rho_amp=0.01)
    u0[:, solid == 1] = 0
    rng = np.random.default_rng(94)
    phi = 1.0 + 0.5 * rng.random(N)
    F = lbm.LBM(q, *dims, 0.7, Th, solid=solid, storage="fp64")
    F.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    S = lbm.ADE(q, *dims, 0.9, ThS, solid=solid, storage="fp64")
    view = S.velocity_view()
    assert view.shape == (2, N) and view.dtype == torch.float64
    S.init(torch.as_tensor(phi))
    for _ in range(25):
        F.step(1)
        F.moments_into(u=view)
        S.step(1)
    phi_g = S.scalar().cpu().numpy()
    Pf = oracle.Problem(q, *dims, 0.7, Th, solid=solid)
    f = Pf.init(rho0, u0)
    g = oracle.ADEProblem(q, *dims, 0.9, ThS, np.zeros((2, N)), solid=solid).init_scalar(phi)
    for _ in range(25):
        Pf.run(f, 1)
        _, uf, _ = Pf.moments(f)
        Ps = oracle.ADEProblem(q, *dims, 0.9, ThS, uf, solid=solid)
        Ps.run_scalar(g, 1)
    assert np.abs(phi_g - Ps.scalar(g)).max() < 1e-13


@pytest.mark.parametrize("q,dims", [(19, (128, 6, 5)), (9, (256, 12, 1))])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_fp16_four_cell_kernels_match_oracle(q, dims, scheme):
    """Rows that fill warps of four-cell threads (nx a multiple of 128) run the scalar through the
    four-cells-per-thread kernels with the velocity read as aligned float2 pairs: FP16-shifted
    storage against the FP64 oracle, 30 steps."""
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    Th = rand_theta(110 + q, d)
    rng = np.random.default_rng(111 + q)
    phi = 1.0 + 0.3 * rng.random(N)
    u = 0.04 * rng.standard_normal((d, N))
    g = _gpu(q, dims, 0.7, Th, phi.astype(np.float32), u.astype(np.float32), 30, storage="fp16s", scheme=scheme)
    P = oracle.ADEProblem(q, *dims, 0.7, Th, u.astype(np.float32).astype(np.float64))
    go = P.init_scalar(phi.astype(np.float32).astype(np.float64))
    P.run_scalar(go, 30)
    err = rel_l2(g["phi"] - 1.0, P.scalar(go) - 1.0)
    print(f"D{d}Q{q} {scheme}: rel (phi - 1) L2 = {err:.3e}")
    assert err < 1e-3


def test_graph_replay_and_state_roundtrip_bit_exact():
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims = 27, (29, 14, 11)
    N = int(np.prod(dims))
    Th = rand_theta(95, 3)
    solid = inputs.random_mask(N, 0.15, 96)
    rng = np.random.default_rng(97)
    phi = 1.0 + 0.3 * rng.random(N)
    u = 0.04 * rng.standard_normal((3, N))
    for storage in ("fp32", "fp16s"):
        for scheme in ("pull", "aa"):
            runs = []
            for graphs in (1, -1):
                A = lbm.ADE(q, *dims, 0.65, Th, u=u, solid=solid, storage=storage, scheme=scheme,
                            use_graphs=graphs)
                A.init(torch.as_tensor(phi))
                A.step(37)
                runs.append(A.populations().cpu())
            assert torch.equal(runs[0], runs[1])
            A.step(0)
            st = A.get_state()
            A.step(9)
            fa = A.populations().cpu()
            B = lbm.ADE(q, *dims, 0.65, Th, u=u, solid=solid, storage=storage, scheme=scheme)
            B.set_state(st)
            assert B.steps == 37
            B.step(9)
            assert torch.equal(fa, B.populations().cpu())
            F = lbm.LBM(q, *dims, 0.65, Th, solid=solid, storage=storage, scheme=scheme)
            with pytest.raises(lbm.LBMError) as e:  # a scalar state does not restore into a flow
                F.set_state(st)
            assert e.value.status == -1


def test_scalar_error_paths():
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims = 19, (16, 8, 8)
    N = int(np.prod(dims))
    A = lbm.ADE(q, *dims, 0.7, np.eye(3) / 3, storage="fp64")
    with pytest.raises(lbm.LBMError) as e:
        A.step(1)
    assert e.value.status == -9
    phi = np.zeros(N)  # phi <= 0 is a valid scalar state
    phi[5] = -0.5
    A.init(torch.as_tensor(phi))
    A.step(3)
    tot, _ = A.totals()
    assert abs(tot + 0.5) < 1e-12
    with pytest.raises(lbm.LBMError) as e:  # init takes no velocity
        from paper_2605_27004_gb300.lbm import _check, _ptr
        u = torch.zeros(3, N, device="cuda", dtype=torch.float64)
        _check(lbm.load().lbm_init(A.ctx, None, _ptr(u)), A.ctx)
    assert e.value.status == -1
    with pytest.raises(lbm.LBMError) as e:
        A.adjoint(torch.zeros(3, N), 3)
    assert e.value.status == -1
    with pytest.raises(lbm.LBMError) as e:
        A.record_checkpoints(2)
    assert e.value.status == -1
    with pytest.raises(lbm.LBMError) as e:
        A.gradients()
    assert e.value.status == -1
    L = lbm.LBM(q, *dims, 0.7, np.eye(3) / 3)
    with pytest.raises(lbm.LBMError) as e:  # velocity calls on a flow context
        from paper_2605_27004_gb300.lbm import _check
        _check(lbm.load().lbm_ade_set_velocity(L.ctx, None, None), L.ctx)
    assert e.value.status == -1
    bad = np.ones(N)
    bad[17] = np.nan
    C = lbm.ADE(q, *dims, 0.7, np.eye(3) / 3, check_every=2)
    C.init(torch.as_tensor(bad, dtype=torch.float32))
    with pytest.raises(lbm.LBMError) as e:
        C.step(4)
    assert e.value.status == -6
    with pytest.raises(lbm.LBMError) as e:
        C.totals()
    assert e.value.status == -6


def test_full_size_sampled_d3q19_fp32_256():
    """The scalar workload the benchmark times, at full size: D3Q19 FP32 256^3, Taylor-Green
    velocity field (u0 = 0.05), rotated Theta, tau 0.6; every population of 500 sampled cells after
    12 steps recomputed from the oracle's one-cell collision of the source cells."""
    import torch
    from paper_2605_27004_gb300 import lbm
    n, q, tau = 256, 19, 0.6
    N = n ** 3
    Th = inputs.theta_rotated([0.36, 0.33, 0.30], inputs.SEED_BASE + 2)
    k = 2 * np.pi / n
    ax = torch.arange(n, device="cuda", dtype=torch.float32) * k
    s_, c_ = torch.sin(ax), torch.cos(ax)
    u = torch.zeros((3, n, n, n), device="cuda", dtype=torch.float32)
    u[0] = 0.05 * s_[None, None, :] * c_[None, :, None] * c_[:, None, None]
    u[1] = -0.05 * c_[None, None, :] * s_[None, :, None] * c_[:, None, None]
    u = u.reshape(3, N)
    xs_ = torch.arange(n, device="cuda", dtype=torch.float32)
    r2 = ((xs_[None, None, :] - 100) ** 2 + (xs_[None, :, None] - 140) ** 2 + (xs_[:, None, None] - 128) ** 2)
    phi = (1.0 + 0.5 * torch.exp(-r2 / (2 * 20.0 ** 2))).reshape(N)
    A = lbm.ADE(q, n, n, n, tau, Th, u=u, storage="fp32")
    A.init(phi)
    A.step(12)
    ga = A.populations()
    A.step(1)
    gb = A.populations()
    c, _ = lbm.lattice_info(q)
    perm = perm_lib_to_oracle(q)
    inv = np.argsort(perm)
    rng = np.random.default_rng(98)
    xs = rng.integers(0, N, size=500)

    def index(x, y, z):
        return (x % n) + n * ((y % n) + n * (z % n))

    need = sorted({int(index(m % n - c[i, 0], (m // n) % n - c[i, 1], m // (n * n) - c[i, 2]))
                   for m in xs for i in range(q)})
    nd = torch.as_tensor(need, device="cuda")
    ga_s = ga[:, nd].double().cpu().numpy()
    u_s = u[:, nd].double().cpu().numpy()
    gb_s = gb[:, torch.as_tensor(xs, device="cuda")].double().cpu().numpy()
    col = {}
    for j, m in enumerate(need):
        col[m] = oracle.ade_collide_cell(q, ga_s[:, j][inv], u_s[:, j], tau, Th)[perm]
    worst = 0.0
    for j, m in enumerate(xs):
        x, y, z = m % n, (m // n) % n, m // (n * n)
        for i in range(q):
            worst = max(worst, abs(gb_s[i, j] - col[int(index(x - c[i, 0], y - c[i, 1], z - c[i, 2]))][i]))
    print("max |g_gpu - g_oracle| over samples:", worst)
    assert worst < 2e-6

"""Z-slab decomposition on one GPU: slab contexts (z_halo) whose ghost planes are filled by the
halo exchange, against the whole-box context and the FP64 oracle.

Every slab runs the same per-cell kernels as the whole box, so with the same inputs the
populations, moments and du0 of the sharded run are bit-identical to the whole-box run in every
storage form; totals and the Theta / tau gradients are sums over cells whose grouping changes
with the cut (FP64, agreement to round-off). The slabs of one box live on one device here, each
with its own stream and host thread (paper_2605_27004_gb300.slabs.SlabGroup); between processes
the same callbacks exchange over torch.distributed.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

from gpu_util import oracle_run, perm_lib_to_oracle, rand_theta, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


def _whole(q, dims, Th, solid, storage, rho0, u0, steps, tau=0.7):
    import torch
    from paper_2605_27004_gb300 import lbm
    L = lbm.LBM(q, *dims, tau, Th, solid=solid, storage=storage)
    dt = L.dtype
    L.init(torch.as_tensor(rho0, dtype=dt), torch.as_tensor(u0, dtype=dt))
    L.step(steps)
    return L


def _group(q, dims, Th, solid, storage, rho0, u0, steps, nslabs, tau=0.7):
    import torch
    from paper_2605_27004_gb300 import slabs
    G = slabs.SlabGroup(q, *dims, tau, Th, nslabs, solid=solid, storage=storage)
    G.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    G.step(steps)
    return G


CASES = [(19, (20, 9, 12), None, 3), (19, (16, 6, 11), "random", 2), (27, (13, 7, 9), "random", 3),
         (27, (12, 5, 8), None, 4), (19, (10, 4, 7), "walls", 7), (19, (128, 4, 7), None, 3)]


def _mask(dims, kind, seed):
    N = int(np.prod(dims))
    if kind is None:
        return None
    if kind == "random":
        return inputs.random_mask(N, 0.2, seed)
    nx, ny, nz = dims
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, 0] = 1  # walls at y = 0 and y = ny - 1, slabs cut across them
    m[:, -1] = 1
    return m.reshape(-1)


@pytest.mark.parametrize("q,dims,mask,nslabs", CASES)
@pytest.mark.parametrize("storage", ["fp64", "fp32s", "fp16s"])
def test_slabs_match_whole_box_bitwise(q, dims, mask, nslabs, storage):
    import torch
    N = int(np.prod(dims))
    Th = rand_theta(40 + q, 3)
    solid = _mask(dims, mask, 41)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 42 + q, rho_amp=0.02)
    steps = 13
    W = _whole(q, dims, Th, solid, storage, rho0, u0, steps)
    G = _group(q, dims, Th, solid, storage, rho0, u0, steps, nslabs)
    fw, fg = W.populations(), G.populations()
    rw, uw, pw = W.moments(Pi=True)
    rg, ug, pg = G.moments(Pi=True)
    torch.cuda.synchronize()
    assert torch.equal(fw, fg)
    assert torch.equal(rw, rg) and torch.equal(uw, ug) and torch.equal(pw, pg)
    mw, jw = W.totals()
    mg, jg = G.totals()
    assert abs(mg - mw) <= 1e-13 * abs(mw)
    assert np.abs(jg - jw).max() <= 1e-13 * abs(mw)
    assert G.exchanges == steps
    W.close()
    G.close()


@pytest.mark.parametrize("q,dims,mask,nslabs", [(19, (12, 7, 10), "random", 3), (27, (10, 6, 9), None, 2)])
def test_slabs_fp64_match_oracle(q, dims, mask, nslabs):
    N = int(np.prod(dims))
    Th = rand_theta(50 + q, 3)
    solid = _mask(dims, mask, 51)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 52 + q, rho_amp=0.02)
    G = _group(q, dims, Th, solid, "fp64", rho0, u0, 20, nslabs)
    o = oracle_run(q, dims, 0.7, Th, rho0, u0, 20, solid=solid)
    f = G.populations().cpu().numpy()
    f_or = o["f"][:, perm_lib_to_oracle(q)].T
    assert np.abs(f - f_or).max() < 1e-13
    G.close()


def test_single_slab_without_callback_is_the_periodic_box():
    """A z_halo context with no callback fills its ghost planes from its own boundary planes:
    the whole periodic box, bit for bit (pair kernels of FP16 storage included)."""
    import torch
    from paper_2605_27004_gb300 import lbm, slabs
    q, dims = 19, (16, 8, 9)
    N = int(np.prod(dims))
    Th = rand_theta(60, 3)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 61, rho_amp=0.02)
    for storage in ("fp64", "fp16s"):
        W = _whole(q, dims, Th, None, storage, rho0, u0, 9)
        c, _ = lbm.lattice_info(q)
        plan = slabs.HaloPlan(c, dims[2], 1, 0)
        S = lbm.LBM(q, *dims, 0.7, Th, storage=storage, z_halo=True)
        dt = S.dtype
        S.init(slabs.slab_of(torch.as_tensor(rho0, dtype=dt), plan, 16, 8),
               slabs.slab_of(torch.as_tensor(u0, dtype=dt), plan, 16, 8))
        S.step(9)
        f_s = slabs.interior_of(S.populations(), plan, 16, 8).reshape(q, -1)
        assert torch.equal(f_s, W.populations())
        W.close()
        S.close()


def test_distributed_slab_world_one_is_the_periodic_box():
    """The one-slab-per-process class with no process group (world size 1): the exchange is its
    own boundary planes, through the same callback and transport function as with R ranks."""
    import torch
    from paper_2605_27004_gb300 import slabs
    q, dims = 27, (12, 6, 7)
    N = int(np.prod(dims))
    Th = rand_theta(62, 3)
    solid = _mask(dims, "random", 63)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 64, rho_amp=0.02)
    W = _whole(q, dims, Th, solid, "fp64", rho0, u0, 11)
    D = slabs.DistributedSlab(q, *dims, 0.7, Th, solid=solid, storage="fp64")
    D.L.init(slabs.slab_of(torch.as_tensor(rho0), D.plan, 12, 6), slabs.slab_of(torch.as_tensor(u0), D.plan, 12, 6))
    D.L.step(11)
    assert torch.equal(slabs.interior_of(D.L.populations(), D.plan, 12, 6).reshape(q, -1), W.populations())
    m, j = D.totals()
    mw, jw = W.totals()
    assert abs(m - mw) <= 1e-13 * mw and np.abs(j - jw).max() <= 1e-13 * mw
    W.close()
    D.L.close()


@pytest.mark.parametrize("storage,q,dims,nslabs,mask", [("fp64", 19, (12, 6, 9), 3, "random"),
                                                       ("fp64", 27, (10, 5, 8), 2, None),
                                                       ("fp32s", 19, (14, 6, 10), 2, None)])
def test_slab_adjoint_matches_whole_box(storage, q, dims, nslabs, mask):
    """The adjoint of the sharded run (reverse halo exchange of lambda after every adjoint step,
    forward recompute with the population exchange) gives the whole box's gradients: du0 bit for
    bit, dTheta and dtau to FP64 round-off (their cell sums are grouped by slab)."""
    import torch
    N = int(np.prod(dims))
    Th = rand_theta(70 + q, 3)
    solid = _mask(dims, mask, 71)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 72 + q, rho_amp=0.02)
    steps, K = 12, 4
    W = _whole(q, dims, Th, solid, storage, rho0, u0, steps)
    G = _group(q, dims, Th, solid, storage, rho0, u0, steps, nslabs)
    g = torch.as_tensor(np.random.default_rng(73).standard_normal((3, N)), dtype=W.dtype, device="cuda")
    W.adjoint(g, steps, K)
    G.adjoint(g, steps, K)
    dw, tw, uw = W.gradients()
    dg, tg, ug = G.gradients()
    assert torch.equal(uw, ug)
    assert np.abs(dg - dw).max() <= 1e-12 * np.abs(dw).max()
    assert abs(tg - tw) <= 1e-12 * abs(tw)
    W.close()
    G.close()


def test_halo_pack_matches_the_plan():
    """lbm_halo_pack writes, for each side and kind, the planes and directions the host plan
    names (the array handed to the callback viewed as [q][nz + 2][ny][nx])."""
    import torch
    from paper_2605_27004_gb300 import lbm, slabs
    q, dims = 27, (9, 5, 6)
    N = int(np.prod(dims))
    Th = rand_theta(80, 3)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 81, rho_amp=0.02)
    c, _ = lbm.lattice_info(q)
    plan = slabs.HaloPlan(c, dims[2], 1, 0)
    seen = []

    def halo(kind, array):
        n_all = q * 9 * 5 * (6 + 2)
        view = torch.as_tensor(lbm._FieldView(array, (n_all,), "<f8", S), device="cuda").clone()
        arr = view.reshape(q, 8, 5, 9).cpu().numpy()
        for side in (0, 1):
            buf = torch.empty(S.halo_bytes(kind) // 8, dtype=torch.float64, device="cuda")
            S.halo_pack(kind, side, array, buf)
            torch.cuda.synchronize()
            got = buf.cpu().numpy().reshape(-1, 5, 9)
            seen.append(np.array_equal(got, plan.pack(kind, side, arr)))
            S.halo_unpack(kind, 1 - side, array, buf)  # the slab is its own neighbour

    S = lbm.LBM(q, *dims, 0.7, Th, storage="fp64", z_halo=True, halo=halo)
    S.init(slabs.slab_of(torch.as_tensor(rho0), plan, 9, 5), slabs.slab_of(torch.as_tensor(u0), plan, 9, 5))
    S.step(2)
    S.adjoint(torch.zeros(3, S.N, dtype=torch.float64, device="cuda") + 1e-3, 2, 1)
    assert len(seen) >= 8 and all(seen)
    S.close()


def test_halo_callback_failure_is_reported():
    """A callback that fails stops lbm_step with LBM_ERR_HALO and the Python exception as cause;
    the context is still usable afterwards (nothing faulted on the device)."""
    import torch
    from paper_2605_27004_gb300 import lbm

    calls = []

    def halo(kind, array):
        calls.append(kind)
        if len(calls) == 3:
            raise ValueError("planted failure")

    S = lbm.LBM(19, 8, 4, 5, 0.7, np.eye(3) / 3, z_halo=True, halo=halo)
    S.init()
    with pytest.raises(lbm.LBMError) as e:
        S.step(5)
    assert e.value.status == -10 and isinstance(e.value.__cause__, ValueError)
    S.step(1)
    S.sync()
    S.close()


def test_slab_options_are_validated():
    from paper_2605_27004_gb300 import lbm
    with pytest.raises(lbm.LBMError):
        lbm.LBM(9, 8, 8, 1, 0.7, np.eye(2) / 3, z_halo=True)          # 2D
    with pytest.raises(lbm.LBMError):
        lbm.LBM(19, 8, 8, 4, 0.7, np.eye(3) / 3, z_halo=True, scheme="aa")
    with pytest.raises(lbm.LBMError):
        lbm.ADE(19, 8, 8, 4, 0.7, np.eye(3) / 3, z_halo=True)
    with pytest.raises(lbm.LBMError):
        lbm.LBM(19, 8, 8, 4, 0.7, np.eye(3) / 3, halo=lambda k, a: None)  # callback without z_halo

"""GPU discrete adjoint against the oracle's FP64 adjoint (itself pinned by finite differences).

The loss gradient dL/du(T) is a fixed seeded field g, so the adjoint of both sides is the
gradient of L = sum g.u(T). FP64 storage must agree to 1e-10 relative; FP32 to 1e-3.
"""
import numpy as np
import pytest

import oracle
from paper_2605_27004_gb300 import inputs

from gpu_util import rand_theta, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_27004_gb300 import build
    build.build()


def _run(q, dims, solid, storage, scheme, K, steps, order=3, seed=0):
    import torch
    from paper_2605_27004_gb300 import lbm
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    Th = rand_theta(50 + q + seed, d, 0.03)
    tau = 0.7
    rho0, u0 = inputs.noise_field(N, d, 0.04, 60 + q + seed, rho_amp=0.02)
    rng = np.random.default_rng(70 + q + seed)
    g = rng.standard_normal((d, N))
    if solid is not None:
        u0 = u0 * (1 - solid)[None, :]
        g = g * (1 - solid)[None, :]
    L = lbm.LBM(q, *dims, tau, Th, solid=solid, storage=storage, scheme=scheme, order=order)
    L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    L.step(steps)
    L.adjoint(torch.as_tensor(g), steps, K)
    dth, dtau, du0 = L.gradients()
    pb = oracle.Problem(q, *dims, tau, Th, solid=solid, order=order)
    odth, odtau, odu0 = pb.adjoint(rho0, u0, steps, g)
    return dth, dtau, du0.double().cpu().numpy(), odth, odtau, odu0


@pytest.mark.parametrize("q,dims", [(9, (37, 21, 1)), (19, (21, 12, 9)), (27, (19, 11, 8))])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("mask", [False, True])
@pytest.mark.parametrize("K", [1, 4, 0])
def test_adjoint_fp64_matches_oracle(q, dims, scheme, mask, K):
    N = int(np.prod(dims))
    solid = inputs.random_mask(N, 0.2, 80 + q) if mask else None
    steps = 11
    dth, dtau, du0, odth, odtau, odu0 = _run(q, dims, solid, "fp64", scheme, K, steps)
    assert np.abs(dth - odth).max() <= 1e-10 * np.abs(odth).max()
    assert abs(dtau - odtau) <= 1e-10 * abs(odtau)
    assert rel_l2(du0, odu0) < 1e-10


@pytest.mark.parametrize("order", [2, 3])
def test_adjoint_order2_fp64(order):
    dth, dtau, du0, odth, odtau, odu0 = _run(19, (16, 10, 7), None, "fp64", "pull", 3, 9, order=order)
    assert np.abs(dth - odth).max() <= 1e-10 * np.abs(odth).max()
    assert abs(dtau - odtau) <= 1e-10 * abs(odtau)
    assert rel_l2(du0, odu0) < 1e-10


@pytest.mark.parametrize("storage", ["fp32", "fp32s", "fp16s"])
def test_adjoint_reduced_precision(storage):
    """FP32 adjoint (FP64 gradient accumulation) against the FP64 oracle adjoint on 24^3, 60 steps."""
    q, dims = 19, (24, 24, 24)
    dth, dtau, du0, odth, odtau, odu0 = _run(q, dims, None, storage, "pull", 10, 60)
    print(storage, np.abs(dth - odth).max() / np.abs(odth).max(), abs(dtau - odtau) / abs(odtau), rel_l2(du0, odu0))
    assert np.abs(dth - odth).max() <= 1e-3 * np.abs(odth).max()
    assert rel_l2(du0, odu0) < 1e-3
    # dL/dtau weighs the non-equilibrium part f - feq, which decays to a small fraction of f as
    # the seeded noise relaxes. FP16 storage rounds f - r to 11 bits and plain FP32 storage
    # rounds f ~ 0.3 to ~2e-8 absolute; both are visible against f - feq late in the run. The
    # adjoint differentiates the stored trajectory, so the gap is the forward precision, not the
    # adjoint; the shifted FP32 form keeps 1e-3.
    tol_tau = {"fp32s": 1e-3, "fp32": 1e-2, "fp16s": 5e-2}[storage]
    assert abs(dtau - odtau) <= tol_tau * abs(odtau)


@pytest.mark.parametrize("q,dims,scheme", [(19, (24, 24, 24), "aa"), (19, (30, 14, 10), "pull"),
                                           (9, (40, 34, 1), "pull"), (9, (40, 34, 1), "aa")])
def test_adjoint_fp16_two_cell_kernel(q, dims, scheme):
    """FP16-shifted storage without walls and with even nx runs the two-cells-per-thread adjoint
    kernel (all three layouts of the stored state: pull, AA even and AA odd steps): against the
    FP64 oracle adjoint with the FP16 tolerances of test_adjoint_reduced_precision."""
    dth, dtau, du0, odth, odtau, odu0 = _run(q, dims, None, "fp16s", scheme, 10, 40)
    print(q, scheme, np.abs(dth - odth).max() / np.abs(odth).max(), abs(dtau - odtau) / abs(odtau),
          rel_l2(du0, odu0))
    assert np.abs(dth - odth).max() <= 1e-3 * np.abs(odth).max()
    assert rel_l2(du0, odu0) < 1e-3
    assert abs(dtau - odtau) <= 5e-2 * abs(odtau)


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_recorded_and_host_checkpoints_give_identical_gradients(scheme):
    """Checkpoints recorded during the forward run, taken by the adjoint's own forward pass, or
    kept in pinned host memory all feed the same kernels in the same order: bit-identical."""
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims, steps, K = 19, (20, 12, 10), 23, 5
    N = int(np.prod(dims))
    Th = rand_theta(91, 3, 0.03)
    rho0, u0 = inputs.noise_field(N, 3, 0.04, 92, rho_amp=0.01)
    g = torch.as_tensor(np.random.default_rng(93).standard_normal((3, N)), dtype=torch.float32)
    SB = 19 * N * 4
    out = []
    for mode in ("recorded", "own", "host", "recorded_host"):
        # host: the limit leaves room for the K segment states and at most one checkpoint, so the
        # restores are synchronous; recorded_host: recording keeps one checkpoint on the device
        # (it reserves 2 ceil(sqrt K) + 1 = 7 states), the other four go to host memory, and the
        # flat plan (5 states) leaves one state for restoring them one segment ahead of use
        limit = {"host": (K + 1) * SB, "recorded_host": 8 * SB}.get(mode, 0)
        L = lbm.LBM(q, *dims, 0.7, Th, storage="fp32", scheme=scheme, adjoint_mem_limit=limit)
        if mode.startswith("recorded"):
            L.record_checkpoints(K)
        L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
        L.step(steps)
        L.adjoint(g, steps, K)
        k2, prefetched = L.adjoint_info()
        assert k2 == K
        assert prefetched == (4 if mode == "recorded_host" else 0), mode
        dth, dtau, du0 = L.gradients()
        out.append((dth, dtau, du0.cpu()))
        # a second call reuses the kept working set; a call after releasing it allocates anew
        L.adjoint(g, steps, K)
        out.append(tuple(x.cpu() if hasattr(x, "cpu") else x for x in L.gradients()))
        L.adjoint_release()
        L.adjoint(g, steps, K)
        out.append(tuple(x.cpu() if hasattr(x, "cpu") else x for x in L.gradients()))
        L.close()
    for dth, dtau, du0 in out[1:]:
        assert np.array_equal(dth, out[0][0]) and dtau == out[0][1] and torch.equal(du0, out[0][2])


@pytest.mark.parametrize("scheme,recorded,limits", [("pull", False, (0, 6, 9)), ("aa", True, (0, 6, 8, 9, 11))])
def test_two_level_segments_match_flat(scheme, recorded, limits):
    """When K segment states do not fit (adjoint_mem_limit), a segment is recomputed in
    sub-segments: the first pass keeps the sub-segment starts and the states of the last one,
    the others are recomputed into its buffers. The states and the kernel order are the same
    as in the flat plan, so the gradients are bit-identical. Over recorded checkpoints every
    state buffer that fits is used (limits of 6, 8, 9 and 11 states give 5, 6, 7 and 8 working
    buffers: sub-segments (4, 4, 4), (6, 6), (5, 7) and (4, 8) of K = 12)."""
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims, steps, K = 27, (18, 12, 10), 29, 12
    N = int(np.prod(dims))
    Th = rand_theta(95, 3, 0.03)
    solid = inputs.random_mask(N, 0.15, 96)
    rho0, u0 = inputs.noise_field(N, 3, 0.04, 97, rho_amp=0.01)
    u0 *= (1 - solid)[None, :]
    g = torch.as_tensor(np.random.default_rng(98).standard_normal((3, N)) * (1 - solid)[None, :], dtype=torch.float32)
    SB = q * N * 4
    out = []
    longest = []
    for limit in limits:
        L = lbm.LBM(q, *dims, 0.7, Th, solid=solid, storage="fp32", scheme=scheme, adjoint_mem_limit=limit * SB)
        if recorded:
            L.record_checkpoints(K)
        L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
        L.step(steps)
        for _ in range(2):  # the second call reuses the kept buffers
            L.adjoint(g, steps, K)
            dth, dtau, du0 = L.gradients()
            out.append((dth, dtau, du0.cpu()))
        longest.append(L.adjoint_info()[0])
        L.close()
    for dth, dtau, du0 in out[1:]:
        assert np.array_equal(out[0][0], dth) and out[0][1] == dtau and torch.equal(out[0][2], du0)
    assert longest[0] == K and all(k < K for k in longest[1:])
    if recorded:
        assert longest == [12, 4, 6, 7, 8]
    with pytest.raises(lbm.LBMError) as e:   # even the two-level plan needs 6 states for K = 12
        L = lbm.LBM(q, *dims, 0.7, Th, solid=solid, storage="fp32", scheme=scheme, adjoint_mem_limit=5 * SB)
        L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
        L.step(steps)
        L.adjoint(g, steps, K)
    assert e.value.status == -4


@pytest.mark.parametrize("storage,scheme", [("fp64", "pull"), ("fp16s", "aa"), ("fp32s", "pull")])
def test_segment_graphs_match_launch_by_launch(storage, scheme):
    """Boxes up to 2M cells replay each full adjoint segment as a CUDA graph (K even, device
    checkpoints); use_graphs = -1 launches every kernel from the host. Same kernels, same order:
    bit-identical gradients, and the graph path issues the same number of kernels."""
    import torch
    from paper_2605_27004_gb300 import lbm
    q, dims, steps, K = 19, (32, 18, 14), 46, 8  # five full segments and a partial one
    N = int(np.prod(dims))
    Th = rand_theta(91, 3, 0.03)
    rho0, u0 = inputs.noise_field(N, 3, 0.04, 92, rho_amp=0.02)
    g = torch.as_tensor(np.random.default_rng(93).standard_normal((3, N)))
    out = []
    for ug in (0, -1):
        L = lbm.LBM(q, *dims, 0.7, Th, storage=storage, scheme=scheme, use_graphs=ug)
        L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
        L.step(steps)
        l0 = L.launches
        L.adjoint(g, steps, K)
        launches = L.launches - l0
        dth, dtau, du0 = L.gradients()
        out.append((dth, dtau, du0, launches))
        L.close()
    (a, b, c, la), (x, y, z, lx) = out
    assert np.array_equal(a, x) and b == y and torch.equal(c, z)
    assert la == lx

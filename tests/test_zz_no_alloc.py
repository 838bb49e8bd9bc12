"""lbm_totals_noalloc, the totals entry point for callers that cannot allocate device memory
(its partial sums live in a fixed array inside the library), against lbm_totals.

It runs through the C ABI on cuda:0, twice in a row (the shared array keeps the previous call's
records, which must not leak into the next result). This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    return lbm.load()


@pytest.mark.parametrize("q,dims,storage,rtol", [
    (19, (40, 24, 18), "fp32s", 1e-6),  # lbm_totals sums per-cell FP32 moments, this sums FP32 f in FP64
    (27, (23, 17, 12), "fp64", 1e-12),
    (9, (70, 37, 1), "fp64", 1e-12),
])
def test_totals_noalloc_matches_lbm_totals(lib, q, dims, storage, rtol):
    import torch
    from paper_2605_27004_gb300 import lbm
    d = 2 if q == 9 else 3
    N = int(np.prod(dims))
    solid = inputs.random_mask(N, 0.2, 7)
    rho0, u0 = inputs.noise_field(N, d, 0.05, 8, rho_amp=0.02)
    L = lbm.LBM(q, *dims, 0.7, np.eye(d) / 3 + 0.01, solid=solid, storage=storage)
    L.init(torch.as_tensor(rho0), torch.as_tensor(u0))
    L.step(7)
    mass, mom = L.totals()
    f = L.populations()
    stream = ctypes.c_void_p(L.stream.cuda_stream)
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device=f.device)
        rc = lib.lbm_totals_noalloc(q, *dims, int(storage == "fp64"), ctypes.c_void_p(f.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) <= rtol * abs(mass)
        for a in range(d):
            assert abs(got[1 + a] - mom[a]) <= rtol * abs(mass)
        if d == 2:
            assert got[3] == 0.0


def test_totals_noalloc_rejects_bad_sizes(lib):
    import torch
    buf = torch.zeros(19 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    p, o = ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(out.data_ptr())
    assert lib.lbm_totals_noalloc(19, 2, 2, 0, 0, p, o, None) == -1
    assert lib.lbm_totals_noalloc(9, 2, 2, 2, 0, p, o, None) == -1
    assert lib.lbm_totals_noalloc(19, 65536, 65536, 1, 0, p, o, None) == -1
    assert lib.lbm_totals_noalloc(11, 2, 2, 2, 0, p, o, None) == -1
    # products that exceed 2^63 in 64-bit arithmetic are rejected too, not wrapped to a small N
    assert lib.lbm_totals_noalloc(19, 2 ** 21, 2 ** 21, 2 ** 21, 0, p, o, None) == -1
    big = 2 ** 31 - 1
    assert lib.lbm_totals_noalloc(27, big, big, big, 1, p, o, None) == -1
    assert lib.lbm_totals_noalloc(19, big, 1, 2, 0, p, o, None) == -1

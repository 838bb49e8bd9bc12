"""The porous-medium workload at its full size and step count: D3Q27 512^3, overlapping spheres
(radii 8-16, solid fraction 0.30 of the interior) between solid planes z = 0 and z = 511,
u_x = 0.03 in the fluid, tau 0.7, Theta = diag(0.38, 0.33, 0.29), 2000 steps. The precision of
the two production storage forms, FP32 and FP16-shifted (FP32 arithmetic), is measured against
the library's FP64 mode, which matches the FP64 oracle to 1e-13 per population with walls
(test_gpu_parity); the oracle itself cannot run this box. Reported: relative velocity L2 over
the fluid cells and the relative mass drift, for shifted FP32 (the default), plain FP32,
FP16 shifted by the rest equilibrium r_i, and FP16 shifted by w_i rho0 alone (the comparison form:
at this Theta its stored values carry r_i - w_i rho0 = 9/2 w_i h_i, up to 0.2 w_i)."""
import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_porous_d3q27_512_storage_forms_against_fp64():
    import torch
    from paper_2605_27004_gb300 import lbm
    n, steps = 512, 2000
    solid = inputs.porous_spheres(n, n, n, seed=inputs.SEED_BASE + 3)
    fluid = torch.as_tensor(solid == 0, device="cuda")
    N = n ** 3
    u0 = np.zeros((3, N), dtype=np.float32)
    u0[0] = 0.03 * (1 - solid)
    Th = np.diag([0.38, 0.33, 0.29])
    out = {}
    for storage in ("fp64", "fp32s", "fp32", "fp16s", "fp16w"):
        dt = torch.float64 if storage == "fp64" else torch.float32
        L = lbm.LBM(27, n, n, n, 0.7, Th, solid=solid, storage=storage)
        L.init(None, torch.as_tensor(u0, dtype=dt))
        m0, _ = L.totals()
        L.step(steps)
        m1, _ = L.totals()
        out[storage] = (L.moments(rho=False)[1].double()[:, fluid], (m1 - m0) / m0)
        L.close()
        torch.cuda.empty_cache()
    ref = out["fp64"][0]
    print(f"fp64: mass drift {out['fp64'][1]:.2e}")
    assert abs(out["fp64"][1]) < 1e-12
    errs = {}
    # fp16w measured 6.1e-2 (u) and 1.0e-4 (mass): far outside the FP16 bar, which is the point
    for storage, tol, tol_m in (("fp32s", 1e-5, 1e-6), ("fp32", 1e-5, 1e-6), ("fp16s", 1e-3, 1e-3),
                                ("fp16w", 0.2, 1e-3)):
        u, drift = out[storage]
        err = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
        errs[storage] = err
        print(f"{storage}: relative u L2 {err:.3e}, mass drift {drift:.2e}")
        assert err < tol and abs(drift) < tol_m
    assert errs["fp16w"] > errs["fp16s"]

"""The C-ABI library builds, loads and exports every function include/lbm.h declares; host-side
argument validation answers without touching a GPU (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    return lbm.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_documented_calls():
    names = _declared()
    for required in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_adjoint", "lbm_gradients",
                     "lbm_totals", "lbm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_27004_gb300 import lbm
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in lbm.SIGNATURES, name


def test_lattice_info_pairs_and_weights(lib):
    from paper_2605_27004_gb300 import lbm
    for q in (9, 19, 27):
        c, w = lbm.lattice_info(q)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.all(c[0] == 0)
        for k in range((q - 1) // 2):
            assert np.all(c[2 * k + 1] == -c[2 * k + 2])
        assert len({tuple(v) for v in c}) == q


@pytest.mark.parametrize("theta,tau,code", [
    ([[0.3, 0.1], [0.0, 0.3]], 0.8, -2),      # not symmetric
    ([[0.3, 0.4], [0.4, 0.3]], 0.8, -2),      # indefinite
    ([[0.3, 0.0], [0.0, 0.3]], 0.5, -3),      # tau <= 1/2
    ([[0.3, 0.0], [0.0, float("nan")]], 0.8, -1),
])
def test_create_rejects_bad_parameters(lib, theta, tau, code):
    ctx = ctypes.c_void_p()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rc = lib.lbm_create(ctypes.byref(ctx), 9, 8, 8, 1, tau, th.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == code
    assert not ctx.value


def test_create_rejects_bad_geometry(lib):
    ctx = ctypes.c_void_p()
    th = np.ascontiguousarray(np.eye(3) / 3)
    assert lib.lbm_create(ctypes.byref(ctx), 19, 8, 8, 0, 0.8, th.ctypes.data_as(ctypes.c_void_p), None) == -1
    assert lib.lbm_create(ctypes.byref(ctx), 11, 8, 8, 8, 0.8, th.ctypes.data_as(ctypes.c_void_p), None) == -1
    th2 = np.ascontiguousarray(np.eye(2) / 3)
    assert lib.lbm_create(ctypes.byref(ctx), 9, 8, 8, 2, 0.8, th2.ctypes.data_as(ctypes.c_void_p), None) == -1


def test_status_strings(lib):
    for code in range(-9, 1):
        assert lib.lbm_status_string(code)


@pytest.mark.parametrize("theta,tau,code", [
    ([[0.3, 0.1], [0.0, 0.3]], 0.8, -2),
    ([[0.3, 0.0], [0.0, 0.3]], 0.45, -3),
])
def test_scalar_create_validates_like_flow(lib, theta, tau, code):
    ctx = ctypes.c_void_p()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rc = lib.lbm_ade_create(ctypes.byref(ctx), 9, 8, 8, 1, tau, th.ctypes.data_as(ctypes.c_void_p), None, None)
    assert rc == code
    assert not ctx.value


def test_scalar_calls_reject_null_context(lib):
    p = ctypes.c_void_p()
    assert lib.lbm_ade_set_velocity(None, None, None) == -1
    assert lib.lbm_ade_velocity(None, ctypes.byref(p)) == -1
    assert not p.value


def test_adjoint_plan_calls_reject_null_context(lib):
    k2, pf = ctypes.c_int(7), ctypes.c_int(7)
    assert lib.lbm_adjoint_info(None, ctypes.byref(k2), ctypes.byref(pf)) == -1
    assert (k2.value, pf.value) == (7, 7)
    assert lib.lbm_adjoint_release(None) == -1


def test_default_options_store_shifted_fp32(lib):
    """The default storage is shifted FP32 (f - r_i), the form that meets the FP32 accuracy bar;
    plain FP32 is an explicit option."""
    from paper_2605_27004_gb300 import lbm
    opt = lbm.lbm_options()
    assert lib.lbm_options_default(ctypes.byref(opt)) == 0
    assert opt.storage == lbm.LBM_FP32_SHIFTED
    assert (opt.scheme, opt.order, opt.rho0) == (lbm.LBM_PULL2, 3, 1.0)
    import inspect
    assert inspect.signature(lbm.LBM.__init__).parameters["storage"].default == "fp32s"

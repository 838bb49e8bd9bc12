"""The paper's Taylor-Green experiment (Sec. 4, Fig. 1) on the library, against what the paper
states and against the oracle's linear theory."""
import numpy as np
import pytest

from paper_2605_27004_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def results():
    from paper_2605_27004_gb300 import build
    build.build()
    pytest.importorskip("scipy")
    from paper_2605_27004_gb300.tg2d import experiment
    return experiment()


def test_isotropic_rate_matches_printed_value(results):
    """Sec. 4 prints omega_d = 3.21e-3 (nu (kx^2 + ky^2), 64^2, tau = 1); the fitted rate of the
    isotropic run must round to it (u_max = 0.02 adds only an O(u^2) nonlinear correction)."""
    for r in results:
        if r["A_xy"] == 0.0:
            assert abs(r["omega_fit"] - 3.21e-3) < 0.005e-3, r


def test_second_order_is_blind_to_anisotropy(results):
    """Fig. 1 left: with the second-order equilibrium the rates vary in the fourth decimal only
    (here 3.2149e-3 ... 3.2055e-3, 0.3 %, from the O(u^2) nonlinearity at u_max = 0.02; the
    linear rates are identical), against 31 % for the third order at A~_xy = 0.4."""
    w = np.array([r["omega_fit"] for r in results if r["order"] == 2])
    assert np.ptp(w) < 5e-3 * w.mean()
    assert np.all(np.diff(w) <= 0)  # the paper's zoom also shows the same ordering


def test_third_order_rate_decreases_with_anisotropy(results):
    """Fig. 1 right: with the third-order equilibrium the decay frequency decreases notably as
    A~_xy grows; the fitted rates also bracket the slow and fast shear-mode rates of the linear
    theory of the oracle."""
    from oracle import linear
    rs = [r for r in results if r["order"] == 3]
    w = np.array([r["omega_fit"] for r in rs])
    assert np.all(np.diff(w) < 0)
    assert w[-1] < 0.8 * w[0]
    k = 2 * np.pi / 64
    for r in rs:
        Th = np.array(r["Theta"])
        r1 = linear.shear_rate(9, Th, 1.0, [k, k], [1, -1])
        r2 = linear.shear_rate(9, Th, 1.0, [k, -k], [1, 1])
        assert min(r1, r2) * 0.99 <= r["omega_fit"] <= max(r1, r2) * 1.01

"""Pin of the oracle's discrete adjoint by central finite differences of its forward run.

The loss is L = sum_x g(x).u(x, T) for a fixed seeded g, so dL/du(T) = g. The paper has no
adjoint; the adjoint is the reverse-mode derivative of the LBE of Eq. LBE_BGK started from the
equilibrium, and finite differences of the forward map are the independent reference.
"""
import numpy as np
import pytest

import oracle
from paper_2605_27004_gb300 import inputs

CS2 = 1.0 / 3.0


def _loss(pb, rho0, u0, steps, g):
    _, _, u, _ = pb.simulate(rho0, u0, steps)
    return float((g * u).sum())


def _sym_index(d):
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


CASES = [
    (9, (7, 6, 1), None, 3),
    (9, (6, 5, 1), "walls", 2),
    (19, (5, 4, 4), None, 3),
    (27, (4, 5, 4), "random", 3),
]


@pytest.mark.parametrize("q,dims,mask,order", CASES)
def test_adjoint_matches_finite_differences(q, dims, mask, order):
    nx, ny, nz = dims
    N = nx * ny * nz
    d = oracle.D_OF_Q[q]
    rng = np.random.default_rng(40 + q)
    A = rng.standard_normal((d, d))
    Th = CS2 * np.eye(d) + 0.03 * (A + A.T) / 2
    tau = 0.7
    steps = 12
    solid = None
    if mask == "walls":
        solid = np.zeros((nz, ny, nx), np.uint8)
        solid[:, 0, :] = 1
        solid = solid.reshape(-1)
    elif mask == "random":
        solid = inputs.random_mask(N, 0.2, 41)
    rho0, u0 = inputs.noise_field(N, d, 0.05, 42, rho_amp=0.02)
    if solid is not None:
        u0 = u0 * (1 - solid)[None, :]
    g = rng.standard_normal((d, N))
    if solid is not None:
        g = g * (1 - solid)[None, :]
    pb = oracle.Problem(q, nx, ny, nz, tau, Th, solid=solid, order=order)
    dTh, dtau, du0 = pb.adjoint(rho0, u0, steps, g)

    h = 1e-6
    for k, (a, b) in enumerate(_sym_index(d)):
        E = np.zeros((d, d))
        E[a, b] = E[b, a] = 1.0
        lp = _loss(oracle.Problem(q, nx, ny, nz, tau, Th + h * E, solid, order), rho0, u0, steps, g)
        lm = _loss(oracle.Problem(q, nx, ny, nz, tau, Th - h * E, solid, order), rho0, u0, steps, g)
        fd = (lp - lm) / (2 * h)
        assert abs(dTh[k] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, dTh[k], fd)

    lp = _loss(oracle.Problem(q, nx, ny, nz, tau + h, Th, solid, order), rho0, u0, steps, g)
    lm = _loss(oracle.Problem(q, nx, ny, nz, tau - h, Th, solid, order), rho0, u0, steps, g)
    fd = (lp - lm) / (2 * h)
    assert abs(dtau - fd) <= 1e-7 * max(1.0, abs(fd)), (dtau, fd)

    v = rng.standard_normal((d, N))
    if solid is not None:
        v = v * (1 - solid)[None, :]
    hu = 1e-6
    lp = _loss(pb, rho0, u0 + hu * v, steps, g)
    lm = _loss(pb, rho0, u0 - hu * v, steps, g)
    fd = (lp - lm) / (2 * hu)
    assert abs((du0 * v).sum() - fd) <= 1e-7 * max(1.0, abs(fd)), ((du0 * v).sum(), fd)

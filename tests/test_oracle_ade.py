"""Pins of the oracle's anisotropic advection-diffusion scheme (no GPU).

The paper names the transfer of its equilibrium to advection-diffusion (Sec. 1, Sec. 5) without
equations; the scheme is the flow scheme with rho -> phi and a prescribed velocity, so that
sum geq = phi, sum geq c = phi u, sum geq c c = phi (Theta + u u). What fixes its results:

* the scheme is linear in g, so the cumulants of a concentration blob evolve exactly: with a
  uniform velocity U the mean moves by U per step and, once the non-conserved modes have
  relaxed, the covariance grows by 2 (tau - 1/2) Theta per step (the anisotropic diffusion
  tensor of the Chapman-Enskog limit, Sec. 3 with rho -> phi);
* the total flux obeys J(t+1) = (1 - 1/tau) J(t) + (1/tau) sum_x phi(x, t) u(x) in a periodic
  box, whatever u(x) is (checks that the velocity field is read at the right cell);
* half-way bounce-back at rest on an x-independent, c_x-symmetric state acts as a mirror: a
  channel of H fluid rows equals the periodic box of 2H rows holding the mirrored field;
* the Fourier multiplier of the linear map gives every plane-wave amplitude exactly, and its
  slow eigenvalue tends to the diffusion rate (tau - 1/2) k.Theta.k as k -> 0.
"""
import numpy as np
import pytest

import oracle
from oracle import linear
from paper_2605_27004_gb300 import inputs

CS2 = 1.0 / 3.0
TH2 = np.array([[0.36, 0.05], [0.05, 0.30]])
TH3 = np.array([[0.36, 0.04, 0.02], [0.04, 0.31, -0.03], [0.02, -0.03, 0.33]])


def _theta(d):
    return TH2 if d == 2 else TH3


def _coords(nx, ny, nz):
    n = np.arange(nx * ny * nz)
    return np.stack([n % nx, (n // nx) % ny, n // (nx * ny)]).astype(np.float64)


@pytest.mark.parametrize("q,order", [(9, 2), (9, 3), (19, 3), (27, 2), (27, 3)])
def test_blob_mean_drift_and_covariance_growth(q, order):
    """Mean moves by exactly U per step; covariance grows by exactly 2 (tau - 1/2) Theta."""
    d = oracle.D_OF_Q[q]
    dims = (96, 96, 1) if d == 2 else (48, 48, 48)
    N = int(np.prod(dims))
    tau = 0.8
    U = np.array([0.05, -0.03, 0.02])[:d]
    X = _coords(*dims)[:d]
    c0 = np.array(dims[:d]) / 2 - 0.5
    sig = 5.0 if d == 2 else 2.0
    phi = np.exp(-((X - c0[:, None]) ** 2).sum(0) / (2 * sig * sig))
    P = oracle.ADEProblem(q, *dims, tau, _theta(d), np.tile(U[:, None], (1, N)), order=order)
    g = P.init_scalar(phi)

    def cumulants():
        p = P.scalar(g)
        M = p.sum()
        m1 = (X * p).sum(1) / M
        Y = X - m1[:, None]
        return M, m1, np.einsum("an,bn,n->ab", Y, Y, p) / M

    P.run_scalar(g, 24)  # non-conserved modes decay as (1 - 1/tau)^t = (-1/4)^t
    M0, m0, C0 = cumulants()
    P.run_scalar(g, 1)
    M1, m1, C1 = cumulants()
    assert abs(M1 - M0) < 1e-12 * M0
    assert np.abs(m1 - m0 - U).max() < 1e-10
    assert np.abs(C1 - C0 - 2 * (tau - 0.5) * _theta(d)).max() < 1e-9


@pytest.mark.parametrize("q", [9, 19, 27])
def test_total_flux_relaxes_to_phi_u(q):
    """J(t+1) = (1 - 1/tau) J(t) + (1/tau) sum phi u for a non-uniform velocity field."""
    d = oracle.D_OF_Q[q]
    dims = (20, 14, 1) if d == 2 else (12, 10, 8)
    N = int(np.prod(dims))
    tau = 0.7
    rng = np.random.default_rng(inputs.SEED_BASE + 40)
    u = 0.05 * rng.standard_normal((d, N))
    phi = 1.0 + 0.3 * rng.random(N)
    P = oracle.ADEProblem(q, *dims, tau, _theta(d), u)
    g = P.init_scalar(phi)
    P.run_scalar(g, 3)
    for _ in range(3):
        rho, uu, _ = P.moments(g)
        J0 = (rho * uu).sum(1)
        expect = (1 - 1 / tau) * J0 + (1 / tau) * (rho[None, :] * u).sum(1)
        P.run_scalar(g, 1)
        rho1, uu1, _ = P.moments(g)
        J1 = (rho1 * uu1).sum(1)
        assert np.abs(J1 - expect).max() < 1e-12 * N


@pytest.mark.parametrize("q", [9, 19, 27])
def test_mass_conserved_with_walls_and_field(q):
    d = oracle.D_OF_Q[q]
    dims = (16, 12, 1) if d == 2 else (10, 9, 8)
    N = int(np.prod(dims))
    solid = inputs.random_mask(N, 0.2, inputs.SEED_BASE + 41)
    rng = np.random.default_rng(inputs.SEED_BASE + 42)
    u = 0.04 * rng.standard_normal((d, N))
    phi = 0.5 + rng.random(N)
    P = oracle.ADEProblem(q, *dims, 0.9, _theta(d), u, solid=solid)
    g = P.init_scalar(phi)
    m0 = P.scalar(g).sum()
    P.run_scalar(g, 40)
    assert abs(P.scalar(g).sum() - m0) < 1e-12 * m0
    assert np.all(g[solid.astype(bool)] == 0)


@pytest.mark.parametrize("q", [9, 19, 27])
def test_bounce_back_is_a_mirror_at_rest(q):
    """Walls at the first and last row/plane (normal y in 2D, z in 3D), diagonal Theta, u = 0,
    phi varying along the normal only: the H fluid layers equal those of a periodic box of 2H
    layers with the mirrored profile."""
    d = oracle.D_OF_Q[q]
    H = 10
    Th = np.diag([0.37, 0.30] if d == 2 else [0.37, 0.30, 0.35])
    if d == 2:
        dw, dp = (6, H + 2, 1), (6, 2 * H, 1)
    else:
        dw, dp = (4, 5, H + 2), (4, 5, 2 * H)
    ax = d - 1
    Nw, Np = int(np.prod(dw)), int(np.prod(dp))
    Xw, Xp = _coords(*dw)[ax], _coords(*dp)[ax]
    prof = 1.0 + 0.4 * np.cos(np.arange(H) * 0.9) + 0.1 * np.arange(H) / H
    solid = ((Xw == 0) | (Xw == H + 1)).astype(np.uint8)
    phi_w = np.where(solid == 1, 0.0, prof[np.clip(Xw.astype(int) - 1, 0, H - 1)])
    full = np.concatenate([prof, prof[::-1]])
    phi_p = full[Xp.astype(int)]
    Pw = oracle.ADEProblem(q, *dw, 0.75, Th, np.zeros((d, Nw)), solid=solid)
    Pp = oracle.ADEProblem(q, *dp, 0.75, Th, np.zeros((d, Np)))
    gw = Pw.init_scalar(phi_w)
    gp = Pp.init_scalar(phi_p)
    Pw.run_scalar(gw, 30)
    Pp.run_scalar(gp, 30)
    aw, ap = Pw.scalar(gw), Pp.scalar(gp)
    for layer in range(H):
        assert np.abs(aw[Xw == layer + 1] - ap[Xp == layer]).max() < 1e-13


@pytest.mark.parametrize("q,order", [(9, 3), (19, 2), (27, 3)])
def test_plane_wave_follows_fourier_multiplier(q, order):
    """phi = 1 + eps cos(k.x) with uniform U: every step of the oracle equals G(k)^t exactly."""
    d = oracle.D_OF_Q[q]
    dims = (32, 16, 1) if d == 2 else (16, 8, 8)
    N = int(np.prod(dims))
    m = np.array([3, 1, 2])[:d]
    k = 2 * np.pi * m / np.array(dims[:d])
    U = np.array([0.04, 0.02, -0.03])[:d]
    tau = 0.65
    X = _coords(*dims)[:d]
    phase = k @ X
    P = oracle.ADEProblem(q, *dims, tau, _theta(d), np.tile(U[:, None], (1, N)), order=order)
    g = P.init_scalar(1.0 + 0.01 * np.cos(phase))
    G = linear.ade_amplification(q, _theta(d), tau, k, order, U)
    c, _, _ = oracle.lattice(q)
    ghat = 0.005 * oracle.feq(q, 1.0, U, _theta(d), order)  # the exp(+i k.x) half of the cosine
    for t in range(1, 13):
        P.run_scalar(g, 1)
        ghat = G @ ghat
        amp = (P.scalar(g) * np.exp(-1j * phase)).sum() / N
        assert abs(amp - ghat.sum()) < 1e-14


@pytest.mark.parametrize("q", [9, 19, 27])
def test_slow_rate_tends_to_anisotropic_diffusion(q):
    """-ln|lambda_slow(k)| / (tau - 1/2) k.Theta.k -> 1 with an O(k^2) error, along several
    directions of k (the anisotropy is visible as the spread of the rates)."""
    d = oracle.D_OF_Q[q]
    Th = _theta(d)
    tau = 0.8
    dirs = [np.eye(d)[0], np.eye(d)[1], np.ones(d) / np.sqrt(d)]
    if d == 3:
        dirs.append(np.array([1.0, -1.0, 0.5]) / 1.5)
    for e in dirs:
        errs = []
        for kk in (0.2, 0.1):
            r = linear.ade_decay_rate(q, Th, tau, kk * e)
            errs.append(abs(r / linear.ade_ce_rate(Th, tau, kk * e) - 1))
        assert errs[1] < 4e-3
        assert errs[1] < 0.3 * errs[0] + 1e-9  # second-order convergence in k
    r = [linear.ade_decay_rate(q, Th, tau, 0.05 * e) for e in np.eye(d)]
    expect = [(tau - 0.5) * 0.05 ** 2 * Th[a, a] for a in range(d)]
    assert np.allclose(r, expect, rtol=2e-3)


def test_uniform_state_is_a_fixed_point():
    for q in (9, 19, 27):
        d = oracle.D_OF_Q[q]
        dims = (8, 6, 1) if d == 2 else (6, 5, 4)
        N = int(np.prod(dims))
        U = np.array([0.03, -0.02, 0.01])[:d]
        P = oracle.ADEProblem(q, *dims, 0.7, _theta(d), np.tile(U[:, None], (1, N)))
        g = P.init_scalar(np.full(N, 1.3))
        g0 = g.copy()
        P.run_scalar(g, 5)
        assert np.abs(g - g0).max() < 1e-14


@pytest.mark.parametrize("q,order", [(9, 3), (19, 3), (27, 2)])
def test_one_cell_collision_moments(q, order):
    """g* = g + (geq - g)/tau: phi kept, flux (1 - 1/tau) j + phi u / tau, second moment
    (1 - 1/tau) Pi + phi (Theta + u u) / tau (the equilibrium's moments are exact)."""
    d = oracle.D_OF_Q[q]
    c, _, _ = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    rng = np.random.default_rng(inputs.SEED_BASE + 43)
    g = 0.05 + 0.1 * rng.random(q)
    u = 0.06 * rng.standard_normal(d)
    tau = 0.73
    gs = oracle.ade_collide_cell(q, g, u, tau, _theta(d), order)
    phi = g.sum()
    assert abs(gs.sum() - phi) < 1e-14
    assert np.abs(gs @ cc - ((1 - 1 / tau) * (g @ cc) + phi * u / tau)).max() < 1e-14
    Pi = np.einsum("i,ia,ib->ab", g, cc, cc)
    Ps = np.einsum("i,ia,ib->ab", gs, cc, cc)
    assert np.abs(Ps - ((1 - 1 / tau) * Pi + phi * (_theta(d) + np.outer(u, u)) / tau)).max() < 1e-14
    # one cell with periodic wrap: streaming returns every population to the cell
    P = oracle.ADEProblem(q, 1, 1, 1, tau, _theta(d), u.reshape(d, 1), order=order)
    gg = g.reshape(1, q).copy()
    P.run_scalar(gg, 1)
    assert np.abs(gg[0] - gs).max() < 1e-15

"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it follows. Nothing here compares the oracle with itself: the checks
are printed values (tests/golden), exact quadrature identities, textbook special cases,
conservation laws, brute-force streaming, linear theory and finite differences.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import linear
from paper_2605_27004_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _rand_theta(rng, d, spread=0.04):
    A = rng.standard_normal((d, d))
    return CS2 * np.eye(d) + spread * (A + A.T) / 2


# ------------------------------------------------------------------------------------------
# Lattices (Appendix C)
# ------------------------------------------------------------------------------------------
def test_d1q3_matches_printed_nodes_and_weights():
    nodes, w = oracle.d1q3()
    rows = _golden_rows("d1q3_gauss_hermite.txt")
    for node_mult, weight in rows:
        x = float(node_mult) * math.sqrt(3.0)
        k = int(np.argmin(np.abs(nodes - x)))
        assert abs(nodes[k] - x) < 1e-15
        assert abs(w[k] - float(Fraction(weight))) < 1e-15


@pytest.mark.parametrize("q", [9, 19, 27])
def test_lattice_isotropy(q):
    d = oracle.D_OF_Q[q]
    c, w, opp = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    assert len(set(map(tuple, c))) == q
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ cc).max() < 1e-16
    I = np.eye(d)
    assert np.abs(np.einsum("i,ia,ib->ab", w, cc, cc) - CS2 * I).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ig->abg", w, cc, cc, cc)).max() < 1e-16
    m4 = np.einsum("i,ia,ib,ig,ie->abge", w, cc, cc, cc, cc)
    iso4 = CS2 ** 2 * (np.einsum("ab,ge->abge", I, I) + np.einsum("ag,be->abge", I, I)
                       + np.einsum("ae,bg->abge", I, I))
    assert np.abs(m4 - iso4).max() < 1e-15
    for i in range(q):
        assert np.all(c[opp[i]] == -c[i])


def test_d3q19_weights_match_textbook():
    c, w, _ = oracle.lattice(19)
    c2 = (c ** 2).sum(axis=1)
    for cnorm, count, weight in _golden_rows("d3q19_weights.txt"):
        sel = c2 == int(cnorm)
        assert sel.sum() == int(count)
        assert np.allclose(w[sel], float(Fraction(weight)), rtol=0, atol=1e-16)


# ------------------------------------------------------------------------------------------
# Discrete equilibrium (Eq. 3rd_order_equilibrium, Eq. feq_i) and its moments (Appendix E)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [9, 19, 27])
@pytest.mark.parametrize("order", [2, 3])
def test_equilibrium_moments_exact(q, order):
    """Sum feq = rho, sum feq c = rho u, sum feq cc = rho (Theta + uu) (Eqs. a0discrete,
    a1discrete; second moment of Appendix E with c_s^2 A^{-1} = Theta)."""
    rng = np.random.default_rng(100 + q + order)
    d = oracle.D_OF_Q[q]
    c, w, _ = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    for _ in range(5):
        Th = _rand_theta(rng, d)
        u = rng.uniform(-0.15, 0.15, d)
        rho = rng.uniform(0.8, 1.2)
        f = oracle.feq(q, rho, u, Th, order)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(f @ cc - rho * u).max() < 1e-15
        M2 = np.einsum("i,ia,ib->ab", f, cc, cc)
        assert np.abs(M2 - rho * (Th + np.outer(u, u))).max() < 2e-15


def _third_moment_exact(rho, u, T):
    return rho * (np.einsum("ab,g->abg", T, u) + np.einsum("bg,a->abg", T, u) + np.einsum("ga,b->abg", T, u)
                  + np.einsum("a,b,g->abg", u, u, u))


@pytest.mark.parametrize("q", [9, 27])
def test_third_moment_mixed_components(q):
    """Appendix E (Eq. mom_diff1): M_abg = rho(Theta_ab u_g + Theta_bg u_a + Theta_ga u_b + u_a u_b u_g).
    The tensor-product D1Q3 quadrature integrates each coordinate exactly up to degree 5 (Appendix
    C, N <= 2n - 1), which covers every component in which no index occurs three times; xxx-type
    components need degree 6 and are excluded."""
    rng = np.random.default_rng(7 + q)
    d = oracle.D_OF_Q[q]
    c, _, _ = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    for _ in range(5):
        Th = _rand_theta(rng, d)
        u = rng.uniform(-0.15, 0.15, d)
        rho = rng.uniform(0.8, 1.2)
        f = oracle.feq(q, rho, u, Th, 3)
        M3 = np.einsum("i,ia,ib,ig->abg", f, cc, cc, cc)
        ex = _third_moment_exact(rho, u, Th)
        for a in range(d):
            for b in range(d):
                for g in range(d):
                    if a == b == g:
                        continue
                    assert abs(M3[a, b, g] - ex[a, b, g]) < 2e-15, (a, b, g)


@pytest.mark.parametrize("q", [9, 27])
def test_second_order_truncation_third_moment(q):
    """Eq. mom_diff2: with the second-order equilibrium the third moment carries the isotropic
    c_s^2 delta in place of Theta (mixed components, exact as above). Reading: the printed
    u_a u_b u_g term is absent, since a second-order truncation has no cubic Hermite coefficient;
    Appendix G's closing remark names this O(u^3) error."""
    rng = np.random.default_rng(11 + q)
    d = oracle.D_OF_Q[q]
    c, _, _ = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    Th = _rand_theta(rng, d)
    u = rng.uniform(-0.1, 0.1, d)
    rho = 1.1
    f = oracle.feq(q, rho, u, Th, 2)
    M3 = np.einsum("i,ia,ib,ig->abg", f, cc, cc, cc)
    ex = _third_moment_exact(rho, u, CS2 * np.eye(d)) - rho * np.einsum("a,b,g->abg", u, u, u)
    for a in range(d):
        for b in range(d):
            for g in range(d):
                if not a == b == g:
                    assert abs(M3[a, b, g] - ex[a, b, g]) < 2e-15


@pytest.mark.parametrize("q", [9, 19, 27])
def test_isotropic_reduction_textbook(q):
    """Theta = c_s^2 I gives K = 0 (Eq. K-term): order 2 is the textbook BGK equilibrium
    w rho (1 + 3 uc + 9/2 uc^2 - 3/2 u^2); order 3 adds the isotropic Hermite-3 term
    w rho (9/2)(uc^3 - u^2 uc) (Sec. 2.2, probabilists' H3 of Appendix B)."""
    rng = np.random.default_rng(3 + q)
    d = oracle.D_OF_Q[q]
    c, w, _ = oracle.lattice(q)
    cc = c[:, :d].astype(np.float64)
    for _ in range(4):
        u = rng.uniform(-0.2, 0.2, d)
        rho = rng.uniform(0.8, 1.2)
        uc = cc @ u
        usq = u @ u
        tb2 = w * rho * (1 + 3 * uc + 4.5 * uc ** 2 - 1.5 * usq)
        tb3 = tb2 + w * rho * 4.5 * (uc ** 3 - usq * uc)
        assert np.abs(oracle.feq(q, rho, u, CS2 * np.eye(d), 2) - tb2).max() < 1e-16
        assert np.abs(oracle.feq(q, rho, u, CS2 * np.eye(d), 3) - tb3).max() < 1e-16


# ------------------------------------------------------------------------------------------
# Time stepping (Eq. LBE_BGK), streaming and bounce-back
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("q,dims", [(9, (5, 4, 1)), (19, (4, 3, 5)), (27, (3, 4, 5))])
def test_pure_streaming_brute_force(q, dims):
    """With tau -> infinity the collision vanishes and one step must move every population one
    link: f_i(x + c_i) = f_i(x), periodic wrap (Eq. LBE_BGK with 1/tau = 0)."""
    nx, ny, nz = dims
    N = nx * ny * nz
    d = oracle.D_OF_Q[q]
    c, _, _ = oracle.lattice(q)
    rng = np.random.default_rng(5)
    pb = oracle.Problem(q, nx, ny, nz, 1e15, CS2 * np.eye(d))
    f0 = rng.uniform(0.01, 0.2, size=(N, q))
    f1 = pb.run(f0.copy(), 1)
    for n in range(N):
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        for i in range(q):
            m = ((x + c[i, 0]) % nx) + nx * (((y + c[i, 1]) % ny) + ny * ((z + c[i, 2]) % nz))
            assert abs(f1[m, i] - f0[n, i]) < 1e-13


def test_bounce_back_brute_force():
    """Half-way bounce-back: a population whose link ends in a solid cell returns reversed to
    its own cell after one step (textbook rule; the paper names bounce-back in Sec. 5 only)."""
    q, nx, ny, nz = 19, 4, 4, 5
    N = nx * ny * nz
    c, _, opp = oracle.lattice(q)
    solid = inputs.random_mask(N, 0.3, 9)
    rng = np.random.default_rng(6)
    pb = oracle.Problem(q, nx, ny, nz, 1e15, CS2 * np.eye(3), solid=solid)
    f0 = rng.uniform(0.01, 0.2, size=(N, q)) * (1 - solid)[:, None]
    f1 = pb.run(f0.copy(), 1)
    for n in range(N):
        if solid[n]:
            assert np.all(f1[n] == 0)
            continue
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        for i in range(q):
            m = ((x + c[i, 0]) % nx) + nx * (((y + c[i, 1]) % ny) + ny * ((z + c[i, 2]) % nz))
            if solid[m]:
                assert abs(f1[n, opp[i]] - f0[n, i]) < 1e-13
            else:
                assert abs(f1[m, i] - f0[n, i]) < 1e-13


@pytest.mark.parametrize("q", [9, 19, 27])
def test_uniform_flow_is_fixed_point(q):
    """A uniform equilibrium is invariant: streaming a uniform field is the identity and
    feq(m(feq)) = feq because the discrete moments are exact (Eqs. a0discrete, a1discrete)."""
    d = oracle.D_OF_Q[q]
    nx, ny, nz = (6, 5, 1) if d == 2 else (4, 3, 5)
    N = nx * ny * nz
    rng = np.random.default_rng(8)
    Th = _rand_theta(rng, d)
    rho0, u0 = inputs.uniform_flow(N, d, rng.uniform(-0.05, 0.05, d), 1.03)
    pb = oracle.Problem(q, nx, ny, nz, 0.7, Th)
    f0 = pb.init(rho0, u0)
    f1 = pb.run(f0.copy(), 10)
    assert np.abs(f1 - f0).max() < 2e-14  # 10 steps of FP64 rounding on O(0.3) values


@pytest.mark.parametrize("q", [9, 19, 27])
def test_conservation_periodic(q):
    """Mass and momentum are conserved by the BGK LBE on a periodic lattice (Sec. 3, continuity
    and momentum balance; Eqs. Dfzero0, Dfzero1)."""
    d = oracle.D_OF_Q[q]
    nx, ny, nz = (12, 10, 1) if d == 2 else (6, 5, 4)
    N = nx * ny * nz
    rng = np.random.default_rng(12)
    Th = _rand_theta(rng, d)
    rho0, u0 = inputs.noise_field(N, d, 0.05, 13, rho_amp=0.02)
    pb = oracle.Problem(q, nx, ny, nz, 0.62, Th)
    f = pb.init(rho0, u0)
    m0, p0 = pb.totals(f)
    steps = 200
    pb.run(f, steps)
    m1, p1 = pb.totals(f)
    # round-off bound: one ulp-scale error per population per cell per step
    bound = steps * N * q * np.finfo(np.float64).eps * 1.1
    assert abs(m1 - m0) < bound
    assert np.abs(p1 - p0).max() < bound


def test_mass_conservation_with_walls():
    """Half-way bounce-back keeps mass (each population is returned, none is lost)."""
    q, nx, ny, nz = 27, 6, 5, 7
    N = nx * ny * nz
    solid = inputs.random_mask(N, 0.25, 21)
    rho0, u0 = inputs.noise_field(N, 3, 0.05, 22, rho_amp=0.02)
    pb = oracle.Problem(q, nx, ny, nz, 0.7, np.diag([0.38, 0.33, 0.29]), solid=solid)
    f = pb.init(rho0, u0)
    m0, _ = pb.totals(f)
    pb.run(f, 100)
    m1, _ = pb.totals(f)
    assert abs(m1 - m0) < 100 * N * q * np.finfo(np.float64).eps * 1.1


# ------------------------------------------------------------------------------------------
# Decay rates: linear theory, the paper's printed value, Chapman-Enskog
# ------------------------------------------------------------------------------------------
def test_paper_taylor_green_rate():
    """Sec. 4 prints omega_d = 3.21e-3 for 64^2, tau = 1 (isotropic). The analytic value must
    round to it, and the D2Q9 linear rate of the TG shear modes must be within 0.2 % of it."""
    (n, tau, umax, printed), = _golden_rows("taylor_green_2d.txt")
    n, tau, printed = int(n), float(tau), float(printed)
    k = 2 * np.pi / n
    nu = (2 * tau - 1) / 6
    analytic = nu * (k * k + k * k)
    assert round(analytic, 5) == printed
    rate = linear.shear_rate(9, CS2 * np.eye(2), tau, [k, k], [1, -1])
    assert abs(rate - analytic) / analytic < 2e-3


def test_linear_rate_matches_chapman_enskog_shear_wave():
    """Transverse wave along y with u along x: CE rate (tau - 1/2) Theta_yy k^2 (Eq. NSprefinal2);
    the lattice rate differs only by the O(k^2) lattice correction."""
    Th = np.array([[0.36, 0.02], [0.02, 0.30]])
    k = 2 * np.pi / 64
    lin = linear.shear_rate(9, Th, 0.8, [0, k], [1, 0])
    ce = linear.ce_shear_rate(Th, 0.8, [0, k])
    assert abs(ce - 0.3 * 0.30 * k * k) < 1e-18
    assert abs(lin - ce) / ce < 2e-3


@pytest.mark.parametrize("order", [2, 3])
def test_anisotropy_trend_paper_fig1(order):
    """Sec. 4 / Fig. 1: with the 2nd-order equilibrium the TG decay does not respond to A~_xy;
    with the 3rd order the slow mode slows down as A~_xy grows."""
    k = 2 * np.pi / 64
    rates = []
    for axy in (0.0, 0.1, 0.2, 0.4):
        Th = inputs.theta_from_atilde([[1.0, axy], [axy, 1.0]])
        r1 = linear.shear_rate(9, Th, 1.0, [k, k], [1, -1], order=order)
        r2 = linear.shear_rate(9, Th, 1.0, [k, -k], [1, 1], order=order)
        rates.append(min(r1, r2))
    rates = np.array(rates)
    if order == 2:
        assert np.ptp(rates) / rates[0] < 1e-3
    else:
        assert np.all(np.diff(rates) < 0)
        assert rates[-1] < 0.8 * rates[0]


def _fourier_amp(field, coords, k):
    return np.sum(field * np.exp(-1j * (coords @ k))) / field.size


@pytest.mark.parametrize("q,dims,kvec_idx,e", [
    (9, (16, 20, 1), (0, 1, 0), (1, 0, 0)),
    (19, (8, 10, 6), (0, 0, 1), (1, -1, 0)),
    (27, (10, 6, 8), (1, 0, 0), (0, 1, 1)),
])
def test_simulated_decay_matches_linear_theory(q, dims, kvec_idx, e):
    """A small-amplitude transverse wave simulated by the oracle must follow the exact linear
    response of the linearised step (von Neumann analysis of Eq. LBE_BGK)."""
    nx, ny, nz = dims
    d = oracle.D_OF_Q[q]
    N = nx * ny * nz
    n = np.array([nx, ny, nz][:d], dtype=np.float64)
    kint = np.array(kvec_idx[:d], dtype=np.float64)
    k = 2 * np.pi * kint / n
    e = np.array(e[:d], dtype=np.float64)
    e -= k * (k @ e) / (k @ k)
    e /= np.linalg.norm(e)
    rng = np.random.default_rng(31 + q)
    Th = _rand_theta(rng, d, spread=0.03)
    amp = 1e-7
    x, y, z = inputs._grid(nx, ny, nz)
    coords = np.stack([x, y, z][:d], axis=1)
    phase = coords @ k
    u0 = amp * e[:, None] * np.cos(phase)[None, :]
    rho0 = np.ones(N)
    pb = oracle.Problem(q, nx, ny, nz, 0.65, Th)
    t = 60
    f, rho, u, _ = pb.simulate(rho0, u0, t)
    j = rho[None, :] * u
    sim = _fourier_amp(e @ j, coords, k) * 2
    pred = linear.linear_response(q, Th, 0.65, k, e, t, amp=amp)
    assert abs(sim - pred) < 1e-6 * amp


def test_channel_decay_between_bounce_back_walls():
    """Shear mode u_x ~ sin(pi (z - 1/2)/H) between half-way bounce-back walls (solid planes
    z = 0 and z = H + 1, walls half-way at z = 1/2 and H + 1/2): decay rate (tau - 1/2) Theta_zz
    (pi/H)^2 (Eq. NSprefinal2), up to the O(1/H^2) lattice error."""
    H = 24
    nx, ny, nz = 4, 4, H + 2
    N = nx * ny * nz
    tau = 0.8
    Th = np.diag([0.36, 0.33, 0.30])
    solid = inputs.channel_walls(nx, ny, nz)
    x, y, z = inputs._grid(nx, ny, nz)
    u0 = np.zeros((3, N))
    u0[0] = 1e-6 * np.sin(np.pi * (z - 0.5) / H) * (1 - solid)
    rho0 = np.ones(N)
    pb = oracle.Problem(27, nx, ny, nz, tau, Th, solid=solid)
    f = pb.init(rho0, u0)
    prof = np.sin(np.pi * (z - 0.5) / H) * (1 - solid)
    amps = []
    steps = [200, 400]
    done = 0
    for s in steps:
        pb.run(f, s - done)
        done = s
        _, u, _ = pb.moments(f)
        amps.append((u[0] * prof).sum() / (prof * prof).sum())
    rate = -np.log(amps[1] / amps[0]) / (steps[1] - steps[0])
    ce = (tau - 0.5) * Th[2, 2] * (np.pi / H) ** 2
    assert abs(rate - ce) / ce < 0.005  # walls at cell centres would be off by 8 %


# ------------------------------------------------------------------------------------------
# Observables of a feq-initialised state (oracle_moments, oracle_totals): the output layout
# ------------------------------------------------------------------------------------------
def _distinct_theta(d):
    """SPD Theta whose entries all differ, so a swapped component of Pi cannot go unnoticed."""
    if d == 2:
        return np.array([[0.36, 0.021], [0.021, 0.30]])
    return np.array([[0.37, 0.013, -0.027], [0.013, 0.33, 0.041], [-0.027, 0.041, 0.29]])


@pytest.mark.parametrize("q,dims", [(9, (6, 5, 1)), (19, (5, 4, 3)), (27, (4, 5, 3))])
@pytest.mark.parametrize("walls", [False, True])
def test_moments_of_equilibrium_state_in_documented_order(q, dims, walls):
    """At t = 0 every fluid cell holds feq(rho0, u0), whose second moment is rho (Theta + u u)
    (Appendix E, the second moment of the discrete equilibrium with c_s^2 A^{-1} = Theta). The
    oracle's Pi output must give it component by component in the order xx, yy, (zz), xy, (xz,
    yz), and rho, u must return the input fields (Eqs. a0discrete_f, a1discrete_f); solid cells
    report zeros. The expected values come from the inputs, not from the oracle."""
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    rng = np.random.default_rng(7000 + q + 10 * walls)
    Th = _distinct_theta(d)
    rho0 = rng.uniform(0.9, 1.1, N)
    # u components of different size so that a swapped velocity index changes the value
    u0 = rng.uniform(-1.0, 1.0, (d, N)) * np.array([0.05, 0.03, 0.017][:d])[:, None]
    solid = None
    if walls:
        solid = (rng.uniform(size=N) < 0.25).astype(np.uint8)
    pb = oracle.Problem(q, *dims, 0.8, Th, solid=solid)
    f = pb.init(rho0, u0)
    rho, u, Pi = pb.moments(f)
    fluid = np.ones(N, bool) if solid is None else solid == 0
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    assert Pi.shape == (len(pairs), N)
    for k, (a, b) in enumerate(pairs):
        want = rho0 * (Th[a, b] + u0[a] * u0[b])
        assert np.abs(Pi[k][fluid] - want[fluid]).max() < 1e-15, (k, a, b)
    assert np.abs(rho[fluid] - rho0[fluid]).max() < 1e-15
    assert np.abs(u[:, fluid] - u0[:, fluid]).max() < 1e-16
    if solid is not None:
        assert not np.any(Pi[:, ~fluid]) and not np.any(rho[~fluid]) and not np.any(u[:, ~fluid])


@pytest.mark.parametrize("q,dims", [(9, (6, 5, 1)), (19, (5, 4, 3)), (27, (4, 5, 3))])
@pytest.mark.parametrize("walls", [False, True])
def test_totals_of_equilibrium_state(q, dims, walls):
    """Mass and momentum totals of f(0) = feq(rho0, u0) are sum rho0 and sum rho0 u0 over the
    fluid cells (Eqs. a0discrete_f, a1discrete_f summed over the box), per component: the velocity
    components differ in size, so a swapped momentum index fails."""
    d = oracle.D_OF_Q[q]
    N = int(np.prod(dims))
    rng = np.random.default_rng(7100 + q + 10 * walls)
    rho0 = rng.uniform(0.9, 1.1, N)
    u0 = np.abs(rng.uniform(0.2, 1.0, (d, N))) * np.array([0.05, -0.03, 0.017][:d])[:, None]
    solid = (rng.uniform(size=N) < 0.25).astype(np.uint8) if walls else None
    pb = oracle.Problem(q, *dims, 0.8, _distinct_theta(d), solid=solid)
    f = pb.init(rho0, u0)
    mass, mom = pb.totals(f)
    fluid = np.ones(N, bool) if solid is None else solid == 0
    assert mom.shape == (d,)
    assert abs(mass - rho0[fluid].sum()) < 1e-13
    want = (rho0[None, fluid] * u0[:, fluid]).sum(axis=1)
    assert np.abs(mom - want).max() < 1e-15 * N

"""Linear (von Neumann) stability analysis of the oracle's BGK scheme.

TEST INFRASTRUCTURE ONLY. Linearises one time step of the oracle around the rest state
(rho0, u = 0) and gives decay rates of plane-wave modes; these are exact for small amplitudes,
which makes them the pin for simulated shear-wave and Taylor-Green decay.

Construction (Sec. 3 derives the macroscopic limit of the same map):
  collision   f* = f + (feq(m(f)) - f)/tau, m = (rho, j);  linearised: J_C = (1 - 1/tau) I + (1/tau) E M
              with E = d feq / d m at (rho0, 0) and M = d m / d f = [1; c^T];
  streaming   f_i(x + c_i, t+1) = f*_i(x)  ->  in Fourier space  f^(k) <- exp(-i k.c_i) f^*(k);
  one step    G(k) = diag(exp(-i k.c_i)) J_C, decay rate of an eigenmode = -ln|lambda| per step.
E is obtained from the oracle's own equilibrium (``oracle.feq``): the equilibrium is a cubic
polynomial in u, so a two-step Richardson central difference is exact up to rounding.

The Chapman-Enskog rate the paper predicts (Eq. NSprefinal2: kinematic viscosity (tau - 1/2)
times Theta = c_s^2 A^{-1}) for a transverse mode with wavevector k is (tau - 1/2) k.Theta.k.
"""
from __future__ import annotations

import numpy as np

from . import D_OF_Q, feq as _feq, lattice as _lattice


def equilibrium_jacobian(q, Theta, order=3, rho0=1.0):
    """E[i, :] = d feq_i / d(rho, j_1..j_d) at (rho0, j = 0), oracle direction order."""
    d = D_OF_Q[q]
    Theta = np.asarray(Theta, dtype=np.float64).reshape(d, d)
    E = np.zeros((q, 1 + d))

    def f_of_m(rho, j):
        return _feq(q, rho, np.asarray(j) / rho, Theta, order)

    j0 = np.zeros(d)
    # rho-derivative at j = 0: feq(rho, 0) is linear in rho
    h = 1e-2
    E[:, 0] = (f_of_m(rho0 + h, j0) - f_of_m(rho0 - h, j0)) / (2 * h)
    for a in range(d):
        def D(step):
            jp = j0.copy()
            jm = j0.copy()
            jp[a] += step
            jm[a] -= step
            return (f_of_m(rho0, jp) - f_of_m(rho0, jm)) / (2 * step)
        # cubic in j at fixed rho: Richardson removes the only error term
        E[:, 1 + a] = (4.0 * D(h) - D(2 * h)) / 3.0
    return E


def collision_jacobian(q, Theta, tau, order=3, rho0=1.0):
    c, _, _ = _lattice(q)
    d = D_OF_Q[q]
    M = np.vstack([np.ones(q), c[:, :d].T.astype(np.float64)])
    E = equilibrium_jacobian(q, Theta, order, rho0)
    om = 1.0 / tau
    return (1.0 - om) * np.eye(q) + om * E @ M


def amplification(q, Theta, tau, k, order=3, rho0=1.0):
    """One-step amplification matrix G(k) (complex q x q)."""
    c, _, _ = _lattice(q)
    d = D_OF_Q[q]
    k = np.asarray(k, dtype=np.float64).reshape(d)
    phase = np.exp(-1j * (c[:, :d] @ k))
    return phase[:, None] * collision_jacobian(q, Theta, tau, order, rho0)


def slow_modes(q, Theta, tau, k, order=3, rho0=1.0):
    """Eigenvalues and eigenvectors of G(k), sorted by |lambda| (slowest decay first)."""
    G = amplification(q, Theta, tau, k, order, rho0)
    lam, V = np.linalg.eig(G)
    idx = np.argsort(-np.abs(lam))
    return lam[idx], V[:, idx]


def shear_rate(q, Theta, tau, k, e, order=3, rho0=1.0):
    """Decay rate per step of the slow eigenmode whose momentum points most along e."""
    d = D_OF_Q[q]
    c, _, _ = _lattice(q)
    lam, V = slow_modes(q, Theta, tau, k, order, rho0)
    e = np.asarray(e, dtype=np.float64).reshape(d)
    e = e / np.linalg.norm(e)
    best, score = None, -1.0
    for m in range(d + 1):
        j = c[:, :d].T.astype(np.float64) @ V[:, m]
        s = abs(e @ j) / (np.linalg.norm(j) + 1e-300)
        if s > score:
            best, score = m, s
    return float(-np.log(np.abs(lam[best])))


def linear_response(q, Theta, tau, k, e, t, amp=1.0, order=3, rho0=1.0):
    """Complex amplitude of e.j(k) after t steps, starting from the equilibrium of a transverse
    velocity perturbation amp * e * exp(i k.x) at uniform density."""
    d = D_OF_Q[q]
    c, _, _ = _lattice(q)
    E = equilibrium_jacobian(q, Theta, order, rho0)
    e = np.asarray(e, dtype=np.float64).reshape(d)
    m0 = np.zeros(1 + d)
    m0[1:] = rho0 * amp * e
    f0 = E @ m0
    G = amplification(q, Theta, tau, k, order, rho0)
    ft = np.linalg.matrix_power(G, int(t)) @ f0
    j = c[:, :d].T.astype(np.float64) @ ft
    return complex(e @ j) / rho0


def ce_shear_rate(Theta, tau, k):
    """Chapman-Enskog rate (tau - 1/2) k.Theta.k of a transverse mode (Eq. NSprefinal2)."""
    k = np.asarray(k, dtype=np.float64)
    Theta = np.asarray(Theta, dtype=np.float64).reshape(k.size, k.size)
    return float((tau - 0.5) * k @ Theta @ k)


def ade_amplification(q, Theta, tau, k, order=3, u=None):
    """One-step Fourier multiplier of the advection-diffusion scheme (oracle_ade_run) with a
    uniform advecting velocity u. The map is linear in g (u is prescribed and geq is linear in
    phi: geq(phi, u) = phi geq(1, u)), so this is exact, not a linearisation:
    G(k) = diag(exp(-i k.c_i)) [(1 - 1/tau) I + (1/tau) e 1^T] with e = geq(1, u)."""
    c, _, _ = _lattice(q)
    d = D_OF_Q[q]
    Theta = np.asarray(Theta, dtype=np.float64).reshape(d, d)
    u = np.zeros(d) if u is None else np.asarray(u, dtype=np.float64).reshape(d)
    e = _feq(q, 1.0, u, Theta, order)
    om = 1.0 / tau
    J = (1.0 - om) * np.eye(q) + om * np.outer(e, np.ones(q))
    k = np.asarray(k, dtype=np.float64).reshape(d)
    return np.exp(-1j * (c[:, :d] @ k))[:, None] * J


def ade_decay_rate(q, Theta, tau, k, order=3, u=None):
    """Decay rate per step of the slowest (diffusive) eigenmode."""
    lam = np.linalg.eigvals(ade_amplification(q, Theta, tau, k, order, u))
    return float(-np.log(np.abs(lam).max()))


def ade_ce_rate(Theta, tau, k):
    """Anisotropic diffusion rate (tau - 1/2) k.Theta.k of the Chapman-Enskog limit."""
    k = np.asarray(k, dtype=np.float64)
    return float((tau - 0.5) * k @ np.asarray(Theta).reshape(k.size, k.size) @ k)

"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input recipes only (fields, masks, anisotropy tensors); it contains none of
the method's arithmetic and imports neither the CUDA library nor the oracle, so both the tests'
oracle side and the device side draw identical inputs from it. Every generator takes an explicit
seed and returns NumPy float64 arrays in the library's field layout: rho ``(N,)``, u ``(d, N)``
with cell index ``x + nx*(y + ny*z)``, solid mask uint8 ``(N,)`` (1 = solid).
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0
SEED_BASE = 20260527


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64), z.reshape(-1).astype(np.float64)


# --------------------------------------------------------------------------------------------
# Anisotropy tensors
# --------------------------------------------------------------------------------------------
def theta_from_atilde(atilde) -> np.ndarray:
    """Theta = c_s^2 A^{-1} with A = Atilde / det(Atilde)^{1/d} (Sec. 4 normalises A to det 1;
    the 2D case there is A = Atilde / sqrt(det Atilde))."""
    At = np.asarray(atilde, dtype=np.float64)
    d = At.shape[0]
    A = At / np.linalg.det(At) ** (1.0 / d)
    return CS2 * np.linalg.inv(A)


def random_rotation(seed: int, d: int = 3) -> np.ndarray:
    """Haar-like rotation: Q of a QR factorisation of a seeded Gaussian, column signs fixed by
    diag(R) > 0 and det(Q) = +1."""
    rng = np.random.default_rng(seed)
    Qm, Rm = np.linalg.qr(rng.standard_normal((d, d)))
    Qm = Qm * np.sign(np.diag(Rm))[None, :]
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] = -Qm[:, 0]
    return Qm


def theta_rotated(eigs, seed: int) -> np.ndarray:
    """Theta = R diag(eigs) R^T with R = random_rotation(seed)."""
    R = random_rotation(seed, len(eigs))
    return R @ np.diag(np.asarray(eigs, dtype=np.float64)) @ R.T


def theta_spd(seed: int, lo: float = 0.29, hi: float = 0.38, d: int = 3) -> np.ndarray:
    """Seeded SPD Theta with eigenvalues uniform in [lo, hi] and a random orientation."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(lo, hi, size=d)
    R = random_rotation(seed + 1, d)
    return R @ np.diag(lam) @ R.T


# --------------------------------------------------------------------------------------------
# Velocity / density fields
# --------------------------------------------------------------------------------------------
def shear_wave_2d(nx: int = 64, ny: int = 64, amp: float = 0.01, noise: float = 1e-4, seed: int = SEED_BASE + 1):
    """u_x = amp sin(2 pi y / ny) plus uniform noise in [-noise, noise] on both components, rho = 1."""
    x, y, _ = _grid(nx, ny, 1)
    rng = np.random.default_rng(seed)
    N = nx * ny
    u = np.zeros((2, N))
    u[0] = amp * np.sin(2 * np.pi * y / ny)
    if noise:
        u += rng.uniform(-noise, noise, size=(2, N))
    rho = np.ones(N)
    return rho, u


def shear_wave(nx, ny, nz, k_axis: int, u_axis: int, amp: float, d: int = 3):
    """Single transverse sine mode u_{u_axis} = amp sin(2 pi x_{k_axis} / n_{k_axis}), rho = 1."""
    x, y, z = _grid(nx, ny, nz)
    coords = (x, y, z)
    n = (nx, ny, nz)[k_axis]
    N = nx * ny * nz
    u = np.zeros((d, N))
    u[u_axis] = amp * np.sin(2 * np.pi * coords[k_axis] / n)
    return np.ones(N), u


def taylor_green_2d(n: int = 64, umax: float = 0.02, rho0: float = 1.0, p_scale: float = 3.0):
    """2D Taylor-Green vortex of Sec. 4 (Eq. TG_u, Eq. TG_p at t = 0) on an n x n periodic box,
    density rho = rho0 + p_scale * (p - p0) with p0 = 0."""
    x, y, _ = _grid(n, n, 1)
    k = 2 * np.pi / n
    u = np.zeros((2, n * n))
    u[0] = -umax * np.cos(k * x) * np.sin(k * y)
    u[1] = umax * np.cos(k * y) * np.sin(k * x)
    p = -(rho0 * umax ** 2 / 4.0) * (np.cos(2 * k * x) + np.cos(2 * k * y))
    rho = rho0 + p_scale * p
    return rho, u


def taylor_green_3d(n: int, u0: float = 0.02, rho0: float = 1.0):
    """3D Taylor-Green vortex u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0), k = 2 pi/n,
    uniform density rho0."""
    x, y, z = _grid(n, n, n)
    k = 2 * np.pi / n
    u = np.zeros((3, n ** 3))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    return np.full(n ** 3, rho0), u


def random_fourier_modes(n: int, kmax: float = 4.0, amp: float = 0.02, seed: int = SEED_BASE + 4):
    """Solenoidal random field: integer wavevectors 0 < |k| <= kmax with seeded complex Gaussian
    coefficients, projected divergence-free, scaled to max |u| = amp. rho = 1."""
    rng = np.random.default_rng(seed)
    x, y, z = _grid(n, n, n)
    u = np.zeros((3, n ** 3))
    K = int(math.floor(kmax))
    for kx in range(-K, K + 1):
        for ky in range(-K, K + 1):
            for kz in range(-K, K + 1):
                kv = np.array([kx, ky, kz], dtype=np.float64)
                k2 = kv @ kv
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
                a = a - kv * (kv @ a) / k2
                phase = np.exp(1j * (2 * np.pi / n) * (kx * x + ky * y + kz * z))
                u += np.real(a[:, None] * phase[None, :])
    mag = np.sqrt((u ** 2).sum(axis=0)).max()
    u *= amp / mag
    return np.ones(n ** 3), u


def uniform_flow(N: int, d: int, u, rho: float = 1.0):
    uu = np.zeros((d, N))
    for a in range(d):
        uu[a] = u[a]
    return np.full(N, rho), uu


def noise_field(N: int, d: int, amp: float, seed: int, rho_amp: float = 0.0):
    """Uniform random velocity in [-amp, amp] per component; density 1 + U(-rho_amp, rho_amp)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-amp, amp, size=(d, N))
    rho = 1.0 + (rng.uniform(-rho_amp, rho_amp, size=N) if rho_amp else np.zeros(N))
    return rho, u


# --------------------------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------------------------
def porous_spheres(nx: int, ny: int, nz: int, rmin: float = 8.0, rmax: float = 16.0, target: float = 0.30,
                   seed: int = SEED_BASE + 3, walls: bool = True, max_spheres: int = 1000000):
    """Overlapping-sphere porous medium between solid planes z = 0 and z = nz-1.

    Spheres with centres uniform over the box and radii U[rmin, rmax] are added (a cell is solid
    when its centre lies within r of the sphere centre, distances wrapped in x and y) until the
    solid fraction of the interior z in [1, nz-2] first reaches ``target``. Returns uint8 (N,).
    """
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    z_lo, z_hi = (1, nz - 1) if walls else (0, nz)
    n_int = (z_hi - z_lo) * ny * nx
    n_solid = 0
    count = 0
    while n_solid < target * n_int and count < max_spheres:
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        r = rng.uniform(rmin, rmax)
        zs = np.arange(max(0, int(math.floor(cz - r))), min(nz, int(math.ceil(cz + r)) + 1))
        ys = np.arange(int(math.floor(cy - r)), int(math.ceil(cy + r)) + 1)
        xs = np.arange(int(math.floor(cx - r)), int(math.ceil(cx + r)) + 1)
        d2 = ((zs[:, None, None] - cz) ** 2 + (ys[None, :, None] - cy) ** 2 + (xs[None, None, :] - cx) ** 2)
        inside = d2 <= r * r
        yw = np.unique(ys % ny, return_index=True)[1]
        xw = np.unique(xs % nx, return_index=True)[1]
        inside = inside[:, yw][:, :, xw]
        zz, yy, xx = zs, ys[yw] % ny, xs[xw] % nx
        box = solid[np.ix_(zz, yy, xx)]
        new = inside & ~box
        zmask = ((zz >= z_lo) & (zz < z_hi))[:, None, None]
        n_solid += int((new & zmask).sum())
        solid[np.ix_(zz, yy, xx)] = box | inside
        count += 1
    if walls:
        solid[0] = True
        solid[nz - 1] = True
    return solid.reshape(-1).astype(np.uint8)


def channel_walls(nx: int, ny: int, nz: int):
    """Solid planes at z = 0 and z = nz-1, fluid in between."""
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[0] = 1
    solid[nz - 1] = 1
    return solid.reshape(-1)


def random_mask(N: int, frac: float, seed: int):
    rng = np.random.default_rng(seed)
    return (rng.random(N) < frac).astype(np.uint8)

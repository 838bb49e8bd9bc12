"""FP64 CPU oracle for the anisotropic-equilibrium BGK lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg are
the only users. It shares no code with the CUDA library (see ``lbm_oracle.c`` for the method
and for what pins each function). Arrays cross this wrapper as NumPy float64:

* populations ``f``: shape ``(N, q)`` (cell-major), in the oracle's own direction order, whose
  velocities are given by :func:`lattice`;
* fields ``rho``: ``(N,)``; ``u``: ``(d, N)``; ``Pi``: ``(d(d+1)/2, N)`` ordered xx, yy, (zz), xy,
  (xz, yz); cell index ``x + nx*(y + ny*z)``;
* ``solid``: uint8 ``(N,)`` (1 = solid) or ``None``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

D_OF_Q = {9: 2, 19: 3, 27: 3}


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.oracle_d1q3.argtypes = [P, P]
            lib.oracle_lattice.argtypes = [I, P, P, P]
            lib.oracle_lattice.restype = I
            lib.oracle_feq.argtypes = [I, D, P, P, I, P]
            lib.oracle_init.argtypes = [I, I, I, I, P, I, P, P, P, P]
            lib.oracle_run.argtypes = [I, I, I, I, D, P, I, P, P, I]
            lib.oracle_moments.argtypes = [I, I, I, I, P, P, P, P, P]
            lib.oracle_totals.argtypes = [I, I, I, I, P, P, P]
            lib.oracle_adjoint.argtypes = [I, I, I, I, D, P, I, P, P, P, I, P, P, P, P]
            lib.oracle_threads.restype = I
            lib.oracle_collide_cell.argtypes = [I, D, P, I, P, P]
            lib.oracle_collide_cell.restype = I
            lib.oracle_ade_init.argtypes = [I, I, I, I, P, I, P, P, P, P]
            lib.oracle_ade_init.restype = I
            lib.oracle_ade_run.argtypes = [I, I, I, I, D, P, I, P, P, P, I]
            lib.oracle_ade_run.restype = I
            lib.oracle_ade_collide_cell.argtypes = [I, D, P, I, P, P, P]
            lib.oracle_ade_collide_cell.restype = I
            lib.oracle_ade_scalar.argtypes = [I, I, I, I, P, P, P]
            lib.oracle_ade_scalar.restype = I
            for fn in ("oracle_lattice", "oracle_feq", "oracle_init", "oracle_run", "oracle_moments",
                       "oracle_totals", "oracle_adjoint"):
                getattr(lib, fn).restype = I
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(solid, N):
    if solid is None:
        return None
    m = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    if m.size != N:
        raise ValueError("solid mask has the wrong size")
    return m


def threads() -> int:
    return int(_load().oracle_threads())


def d1q3():
    """D1Q3 Gauss-Hermite nodes and weights as the oracle derives them (Appendix C)."""
    nodes = np.zeros(3)
    w = np.zeros(3)
    _load().oracle_d1q3(_ptr(nodes), _ptr(w))
    return nodes, w


def lattice(q: int):
    """(c[q,3] int, w[q], opp[q]) in the oracle's own direction order."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    n = _load().oracle_lattice(q, _ptr(c), _ptr(w), _ptr(opp))
    if n != q:
        raise ValueError(f"unsupported lattice q={q}")
    return c, w, opp


def feq(q: int, rho: float, u, Theta, order: int = 3):
    """Equilibrium of one cell, oracle direction order."""
    d = D_OF_Q[q]
    u = _f64(np.asarray(u).reshape(d))
    Th = _f64(np.asarray(Theta).reshape(d, d))
    out = np.zeros(q)
    if _load().oracle_feq(q, float(rho), _ptr(u), _ptr(Th), int(order), _ptr(out)):
        raise ValueError("oracle_feq failed")
    return out


def collide_cell(q: int, f, tau: float, Theta, order: int = 3):
    """Post-collision populations of one cell (oracle direction order)."""
    d = D_OF_Q[q]
    f = _f64(np.asarray(f).reshape(q))
    Th = _f64(np.asarray(Theta).reshape(d, d))
    out = np.zeros(q)
    if _load().oracle_collide_cell(q, float(tau), _ptr(Th), int(order), _ptr(f), _ptr(out)):
        raise ValueError("oracle_collide_cell failed")
    return out


class Problem:
    """Geometry and parameters of one run (what the library's create call receives)."""

    def __init__(self, q, nx, ny, nz, tau, Theta, solid=None, order=3):
        self.q, self.nx, self.ny, self.nz = int(q), int(nx), int(ny), int(nz)
        self.d = D_OF_Q[self.q]
        self.N = self.nx * self.ny * self.nz
        self.tau = float(tau)
        self.Theta = _f64(np.asarray(Theta).reshape(self.d, self.d))
        self.solid = _mask(solid, self.N)
        self.order = int(order)

    def init(self, rho0, u0):
        f = np.zeros((self.N, self.q))
        rc = _load().oracle_init(self.q, self.nx, self.ny, self.nz, _ptr(self.Theta), self.order,
                                 _ptr(self.solid), _ptr(_f64(rho0).reshape(-1)),
                                 _ptr(_f64(u0).reshape(self.d, self.N)), _ptr(f))
        if rc:
            raise RuntimeError("oracle_init failed")
        return f

    def run(self, f, nsteps):
        """Advance populations ``f`` (modified in place and returned) by ``nsteps``."""
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (self.N, self.q)
        rc = _load().oracle_run(self.q, self.nx, self.ny, self.nz, self.tau, _ptr(self.Theta), self.order,
                                _ptr(self.solid), _ptr(f), int(nsteps))
        if rc:
            raise RuntimeError("oracle_run failed")
        return f

    def moments(self, f):
        np_ = 3 if self.d == 2 else 6
        rho = np.zeros(self.N)
        u = np.zeros((self.d, self.N))
        Pi = np.zeros((np_, self.N))
        rc = _load().oracle_moments(self.q, self.nx, self.ny, self.nz, _ptr(self.solid), _ptr(f), _ptr(rho),
                                    _ptr(u), _ptr(Pi))
        if rc:
            raise RuntimeError("oracle_moments failed")
        return rho, u, Pi

    def totals(self, f):
        out = np.zeros(4)
        _load().oracle_totals(self.q, self.nx, self.ny, self.nz, _ptr(self.solid), _ptr(f), _ptr(out))
        return out[0], out[1:1 + self.d].copy()

    def adjoint(self, rho0, u0, nsteps, dLdu):
        """(dTheta[3|6], dtau, du0[d, N]) for a loss whose gradient w.r.t. u(T) is dLdu."""
        nth = 3 if self.d == 2 else 6
        dTh = np.zeros(nth)
        dtau = np.zeros(1)
        du0 = np.zeros((self.d, self.N))
        rc = _load().oracle_adjoint(self.q, self.nx, self.ny, self.nz, self.tau, _ptr(self.Theta), self.order,
                                    _ptr(self.solid), _ptr(_f64(rho0).reshape(-1)),
                                    _ptr(_f64(u0).reshape(self.d, self.N)), int(nsteps),
                                    _ptr(_f64(dLdu).reshape(self.d, self.N)), _ptr(dTh),
                                    dtau.ctypes.data_as(ctypes.c_void_p), _ptr(du0))
        if rc:
            raise RuntimeError("oracle_adjoint failed")
        return dTh, float(dtau[0]), du0

    def simulate(self, rho0, u0, nsteps):
        """Init + nsteps; returns (f, rho, u, Pi)."""
        f = self.init(rho0, u0)
        self.run(f, nsteps)
        rho, u, Pi = self.moments(f)
        return f, rho, u, Pi


def ade_collide_cell(q: int, g, u, tau: float, Theta, order: int = 3):
    """Post-collision scalar populations of one cell (oracle direction order) for the cell's
    advecting velocity u (see oracle_ade_run)."""
    d = D_OF_Q[q]
    g = _f64(np.asarray(g).reshape(q))
    uu = _f64(np.asarray(u).reshape(d))
    Th = _f64(np.asarray(Theta).reshape(d, d))
    out = np.zeros(q)
    if _load().oracle_ade_collide_cell(q, float(tau), _ptr(Th), int(order), _ptr(g), _ptr(uu), _ptr(out)):
        raise ValueError("oracle_ade_collide_cell failed")
    return out


class ADEProblem(Problem):
    """Anisotropic advection-diffusion of a scalar phi by a fixed velocity field u (see
    oracle_ade_run): same lattice, equilibrium and streaming as the flow problem."""

    def __init__(self, q, nx, ny, nz, tau, Theta, u, solid=None, order=3):
        super().__init__(q, nx, ny, nz, tau, Theta, solid=solid, order=order)
        self.u = _f64(np.asarray(u)).reshape(self.d, self.N)

    def init_scalar(self, phi):
        g = np.zeros((self.N, self.q))
        rc = _load().oracle_ade_init(self.q, self.nx, self.ny, self.nz, _ptr(self.Theta), self.order,
                                     _ptr(self.solid), _ptr(_f64(phi).reshape(-1)), _ptr(self.u), _ptr(g))
        if rc:
            raise RuntimeError("oracle_ade_init failed")
        return g

    def run_scalar(self, g, nsteps):
        assert g.dtype == np.float64 and g.flags.c_contiguous and g.shape == (self.N, self.q)
        rc = _load().oracle_ade_run(self.q, self.nx, self.ny, self.nz, self.tau, _ptr(self.Theta), self.order,
                                    _ptr(self.solid), _ptr(self.u), _ptr(g), int(nsteps))
        if rc:
            raise RuntimeError("oracle_ade_run failed")
        return g

    def scalar(self, g):
        phi = np.zeros(self.N)
        _load().oracle_ade_scalar(self.q, self.nx, self.ny, self.nz, _ptr(self.solid), _ptr(g), _ptr(phi))
        return phi

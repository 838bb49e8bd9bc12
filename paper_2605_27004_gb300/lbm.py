"""Thin ctypes binding of ``liblbm.so`` (C ABI in ``include/lbm.h``).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
Device memory is PyTorch's (field buffers are torch CUDA tensors; library-owned buffers are
drawn from torch's caching allocator through the ABI's allocator hooks) and so is the stream
(the current torch stream at construction). There is no CPU fallback: if the library is missing
or no CUDA device is present, the calls raise.

The module-level functions carry the ABI names (``lbm_create`` ...); :class:`LBM` bundles a
context with those calls for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblbm.so")

LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 9, 19, 27
LBM_FP32, LBM_FP64, LBM_FP32_SHIFTED, LBM_FP16_SHIFTED, LBM_FP16_WSHIFTED = 0, 1, 2, 3, 4
LBM_PULL2, LBM_AA = 0, 1
STORAGE = {"fp32": LBM_FP32, "fp64": LBM_FP64, "fp32s": LBM_FP32_SHIFTED, "fp16s": LBM_FP16_SHIFTED,
           "fp16w": LBM_FP16_WSHIFTED}
SCHEME = {"pull": LBM_PULL2, "aa": LBM_AA}
STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID_ARG", -2: "LBM_ERR_NOT_SPD", -3: "LBM_ERR_BAD_TAU",
          -4: "LBM_ERR_OOM", -5: "LBM_ERR_CUDA", -6: "LBM_ERR_UNSTABLE", -7: "LBM_ERR_NO_FORWARD",
          -8: "LBM_ERR_TIMEOUT", -9: "LBM_ERR_STATE", -10: "LBM_ERR_HALO"}
LBM_HALO_POPULATIONS, LBM_HALO_ADJOINT = 0, 1
D_OF_Q = {9: 2, 19: 3, 27: 3}

# Every exported symbol of the ABI (include/lbm.h), with (restype, argtypes).
_P, _I, _D, _S, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_longlong
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
HALO_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class lbm_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("scheme", ctypes.c_int), ("order", ctypes.c_int),
                ("rho0", ctypes.c_double), ("check_every", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("adjoint_mem_limit", ctypes.c_size_t), ("z_halo", ctypes.c_int),
                ("halo", HALO_FN), ("halo_user", ctypes.c_void_p)]


SIGNATURES = {
    "lbm_options_default": (_I, [ctypes.POINTER(lbm_options)]),
    "lbm_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _D, _P, _P]),
    "lbm_create_ex": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _D, _P, _P, ctypes.POINTER(lbm_options)]),
    "lbm_destroy": (None, [_P]),
    "lbm_set_params": (_I, [_P, _D, _P]),
    "lbm_init": (_I, [_P, _P, _P]),
    "lbm_step": (_I, [_P, _I]),
    "lbm_moments": (_I, [_P, _P, _P, _P]),
    "lbm_populations": (_I, [_P, _P]),
    "lbm_totals": (_I, [_P, _P, _P]),
    "lbm_adjoint": (_I, [_P, _P, _I, _I]),
    "lbm_adjoint_release": (_I, [_P]),
    "lbm_adjoint_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lbm_adjoint_plan": (_I, [_I, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I)]),
    "lbm_record_checkpoints": (_I, [_P, _I]),
    "lbm_gradients": (_I, [_P, _P, _P, _P]),
    "lbm_state_bytes": (_I, [_P, ctypes.POINTER(_S)]),
    "lbm_get_state": (_I, [_P, _P, _S]),
    "lbm_set_state": (_I, [_P, _P, _S]),
    "lbm_steps_done": (_I, [_P, ctypes.POINTER(_LL)]),
    "lbm_sync": (_I, [_P]),
    "lbm_lattice_info": (_I, [_I, _P, _P]),
    "lbm_device_bytes": (_I, [_P, ctypes.POINTER(_S)]),
    "lbm_launch_count": (_I, [_P, ctypes.POINTER(_LL)]),
    "lbm_totals_noalloc": (_I, [_I, _I, _I, _I, _I, _P, _P, _P]),
    "lbm_halo_bytes": (_I, [_P, _I, ctypes.POINTER(_S)]),
    "lbm_halo_pack": (_I, [_P, _I, _I, _P, _P]),
    "lbm_halo_unpack": (_I, [_P, _I, _I, _P, _P]),
    "lbm_ade_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _D, _P, _P, ctypes.POINTER(lbm_options)]),
    "lbm_ade_set_velocity": (_I, [_P, _P, _P]),
    "lbm_ade_velocity": (_I, [_P, ctypes.POINTER(_P)]),
    "lbm_status_string": (ctypes.c_char_p, [_I]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None
_lock = threading.Lock()


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load liblbm.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc, ctx=None, owner=None):
    if rc != 0:
        lib = load()
        msg = lib.lbm_last_error(ctx).decode() if ctx else lib.lbm_status_string(rc).decode()
        cause = getattr(owner, "_halo_error", None)
        if cause is not None:
            owner._halo_error = None
            raise LBMError(rc, msg) from cause
        raise LBMError(rc, msg)
    return rc


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def lattice_info(q: int):
    """(c [q,3] int32, w [q]) in the library's direction order."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    n = load().lbm_lattice_info(q, c.ctypes.data_as(_P), w.ctypes.data_as(_P))
    if n != q:
        raise LBMError(n, f"unknown lattice {q}")
    return c, w


def adjoint_plan(length: int, working: int):
    """Sub-segment starts of the adjoint's recompute plan for a segment of `length` steps with
    `working` free state buffers ([0] when flat), or None when no plan fits (lbm_adjoint_plan)."""
    cap = max(1, int(length))
    starts = (ctypes.c_int * cap)()
    count = ctypes.c_int(0)
    rc = load().lbm_adjoint_plan(int(length), int(working), starts, cap, ctypes.byref(count))
    if rc == -4:
        return None
    if rc != 0:
        raise LBMError(rc, f"lbm_adjoint_plan({length}, {working})")
    return [starts[j] for j in range(count.value)]


class _TorchAllocator:
    """Allocator hooks that hand torch caching-allocator blocks to the library."""

    def __init__(self, device, stream):
        torch = _torch()
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=self.stream)
            except Exception:  # out of memory: the library reports LBM_ERR_OOM
                return None
            self.live[int(p)] = nbytes
            return int(p)

        def _free(ptr, user):
            if ptr:
                self.live.pop(int(ptr), None)
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class LBM:
    """One simulation context (``lbm_create_ex`` ... ``lbm_destroy``)."""

    _scalar = False

    def __init__(self, lattice, nx, ny, nz, tau, Theta, solid=None, storage="fp32s", scheme="pull", order=3,
                 rho0=1.0, check_every=0, use_graphs=0, device=None, stream=None, torch_alloc=True,
                 adjoint_mem_limit=0, z_halo=False, halo=None):
        """z_halo: the context is one z-slab of nz interior planes between two ghost planes
        (fields and the mask then span nx*ny*(nz + 2) cells); halo: the exchange callback
        halo(kind, array_ptr) of such a slab, or None for a slab that is the whole box in z."""
        torch = _torch()
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: liblbm runs on the GPU only")
        self.q = int(lattice)
        self.d = D_OF_Q[self.q]
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.z_halo = bool(z_halo)
        self.N = self.nx * self.ny * (self.nz + 2 if self.z_halo else self.nz)
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dtype = torch.float64 if self.storage == LBM_FP64 else torch.float32
        opt = lbm_options()
        lib.lbm_options_default(ctypes.byref(opt))
        opt.storage = self.storage
        opt.scheme = self.scheme
        opt.order = int(order)
        opt.rho0 = float(rho0)
        opt.check_every = int(check_every)
        opt.use_graphs = int(use_graphs)
        opt.stream = ctypes.c_void_p(self.stream.cuda_stream)
        opt.adjoint_mem_limit = int(adjoint_mem_limit)
        opt.z_halo = int(self.z_halo)
        self._halo = None
        self._halo_error = None
        if halo is not None:
            def _cb(ctx, kind, array, user):
                try:
                    halo(int(kind), int(array or 0))
                    return 0
                except BaseException as e:  # reported by the library as LBM_ERR_HALO, re-raised here
                    self._halo_error = e
                    return 1
            self._halo = HALO_FN(_cb)
            opt.halo = self._halo
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(self.device, self.stream)
            opt.alloc = self._alloc.alloc
            opt.free = self._alloc.free
        Th = np.ascontiguousarray(np.asarray(Theta, dtype=np.float64).reshape(self.d, self.d))
        mask = None
        if solid is not None:
            mask = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
            if mask.size != self.N:
                raise ValueError("solid mask must have N entries")
        ctx = _P()
        create = lib.lbm_ade_create if self._scalar else lib.lbm_create_ex
        with torch.cuda.device(self.device):
            _check(create(ctypes.byref(ctx), self.q, self.nx, self.ny, self.nz, float(tau),
                          Th.ctypes.data_as(_P), None if mask is None else mask.ctypes.data_as(_P),
                          ctypes.byref(opt)))
        self.ctx = ctx
        self._opt = opt
        self.tau = float(tau)
        self.Theta = Th
        self.solid = mask

    # -- helpers -------------------------------------------------------------------------------
    def _field(self, x, shape):
        torch = _torch()
        if x is None:
            return None
        if not isinstance(x, torch.Tensor):
            x = torch.as_tensor(np.asarray(x))
        x = x.to(device=self.device, dtype=self.dtype).contiguous()
        if tuple(x.shape) != shape and x.numel() == int(np.prod(shape)):
            x = x.reshape(shape)
        if tuple(x.shape) != shape:
            raise ValueError(f"field has shape {tuple(x.shape)}, expected {shape}")
        return x

    def _empty(self, *shape):
        return _torch().empty(shape, dtype=self.dtype, device=self.device)

    def close(self):
        if getattr(self, "ctx", None):
            load().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls -----------------------------------------------------------------------------
    def set_params(self, tau, Theta):
        Th = np.ascontiguousarray(np.asarray(Theta, dtype=np.float64).reshape(self.d, self.d))
        _check(load().lbm_set_params(self.ctx, float(tau), Th.ctypes.data_as(_P)), self.ctx)
        self.tau, self.Theta = float(tau), Th

    def init(self, rho=None, u=None):
        rho_t = self._field(rho, (self.N,))
        u_t = self._field(u, (self.d, self.N))
        _check(load().lbm_init(self.ctx, _ptr(rho_t), _ptr(u_t)), self.ctx)
        self._keep = (rho_t, u_t)  # the copies are taken on the stream; keep sources alive

    def step(self, n=1):
        _check(load().lbm_step(self.ctx, int(n)), self.ctx, self)

    def moments(self, rho=True, u=True, Pi=False):
        r = self._empty(self.N) if rho else None
        v = self._empty(self.d, self.N) if u else None
        p = self._empty(3 if self.d == 2 else 6, self.N) if Pi else None
        _check(load().lbm_moments(self.ctx, _ptr(r), _ptr(v), _ptr(p)), self.ctx)
        return r, v, p

    def moments_into(self, rho=None, u=None, Pi=None):
        _check(load().lbm_moments(self.ctx, _ptr(rho), _ptr(u), _ptr(Pi)), self.ctx)

    def populations(self):
        f = self._empty(self.q, self.N)
        _check(load().lbm_populations(self.ctx, _ptr(f)), self.ctx)
        return f

    def totals(self):
        m = ctypes.c_double()
        p = np.zeros(3)
        _check(load().lbm_totals(self.ctx, ctypes.byref(m), p.ctypes.data_as(_P)), self.ctx)
        return m.value, p[: self.d].copy()

    def record_checkpoints(self, checkpoint_every):
        _check(load().lbm_record_checkpoints(self.ctx, int(checkpoint_every)), self.ctx)

    def adjoint(self, loss_grad, n, checkpoint_every=0):
        g = self._field(loss_grad, (self.d, self.N))
        _check(load().lbm_adjoint(self.ctx, _ptr(g), int(n), int(checkpoint_every)), self.ctx, self)

    def adjoint_info(self):
        """(sub-segment length, host checkpoints prefetched) of the last adjoint."""
        k2, pf = ctypes.c_int(), ctypes.c_int()
        _check(load().lbm_adjoint_info(self.ctx, ctypes.byref(k2), ctypes.byref(pf)), self.ctx)
        return k2.value, pf.value

    def adjoint_release(self):
        _check(load().lbm_adjoint_release(self.ctx), self.ctx)

    def gradients(self, du0=True):
        dth = np.zeros(3 if self.d == 2 else 6)
        dtau = ctypes.c_double()
        out = self._empty(self.d, self.N) if du0 else None
        _check(load().lbm_gradients(self.ctx, dth.ctypes.data_as(_P), ctypes.byref(dtau), _ptr(out)), self.ctx)
        return dth, dtau.value, out

    def state_bytes(self):
        b = ctypes.c_size_t()
        _check(load().lbm_state_bytes(self.ctx, ctypes.byref(b)), self.ctx)
        return b.value

    def get_state(self):
        torch = _torch()
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _check(load().lbm_get_state(self.ctx, _ptr(buf), buf.numel()), self.ctx)
        return buf

    def set_state(self, buf):
        _check(load().lbm_set_state(self.ctx, _ptr(buf), buf.numel()), self.ctx)

    @property
    def steps(self):
        s = ctypes.c_longlong()
        _check(load().lbm_steps_done(self.ctx, ctypes.byref(s)), self.ctx)
        return s.value

    @property
    def launches(self):
        s = ctypes.c_longlong()
        _check(load().lbm_launch_count(self.ctx, ctypes.byref(s)), self.ctx)
        return s.value

    @property
    def device_bytes(self):
        s = ctypes.c_size_t()
        _check(load().lbm_device_bytes(self.ctx, ctypes.byref(s)), self.ctx)
        return s.value

    def sync(self):
        _check(load().lbm_sync(self.ctx), self.ctx)

    # -- z-slab halo planes (z_halo contexts) ----------------------------------------------------
    def halo_bytes(self, kind):
        b = ctypes.c_size_t()
        _check(load().lbm_halo_bytes(self.ctx, int(kind), ctypes.byref(b)), self.ctx)
        return b.value

    def halo_pack(self, kind, side, array, buf):
        """Pack the boundary plane for the neighbour on `side` of the device array at address
        `array` (the callback's argument) into the tensor `buf`."""
        _check(load().lbm_halo_pack(self.ctx, int(kind), int(side), ctypes.c_void_p(array), _ptr(buf)), self.ctx)

    def halo_unpack(self, kind, side, array, buf):
        _check(load().lbm_halo_unpack(self.ctx, int(kind), int(side), ctypes.c_void_p(array), _ptr(buf)), self.ctx)


class _FieldView:
    """A library-owned device buffer exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, shape, typestr, owner):
        self._owner = owner  # keeps the context (and with it the buffer) alive
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class ADE(LBM):
    """Anisotropic advection-diffusion of a scalar (``lbm_ade_create``): same constructor
    arguments as :class:`LBM` (``rho0`` is the reference phi0 of the shifted storage) plus the
    advecting velocity ``u`` ([d, N] field, a length-d constant, or None for u = 0)."""

    _scalar = True

    def __init__(self, lattice, nx, ny, nz, tau, Theta, u=None, **kw):
        super().__init__(lattice, nx, ny, nz, tau, Theta, **kw)
        if u is not None:
            self.set_velocity(u)

    def set_velocity(self, u=None):
        """u: [d, N] field (tensor / array), a length-d constant, or None (u = 0)."""
        lib = load()
        if u is None:
            _check(lib.lbm_ade_set_velocity(self.ctx, None, None), self.ctx)
            return
        torch = _torch()
        if (u.numel() if isinstance(u, torch.Tensor) else np.asarray(u).size) == self.d:
            a = u.detach().cpu().numpy() if isinstance(u, torch.Tensor) else u
            cst = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.d))
            _check(lib.lbm_ade_set_velocity(self.ctx, None, cst.ctypes.data_as(_P)), self.ctx)
            return
        t = self._field(u, (self.d, self.N))
        _check(lib.lbm_ade_set_velocity(self.ctx, _ptr(t), None), self.ctx)
        self._keep_u = t  # copied on the context's stream

    def velocity_view(self):
        """The context-owned advecting-velocity field as a [d, N] tensor aliasing it (write into
        it to change the velocity between steps, e.g. ``flow.moments_into(u=ade.velocity_view())``)."""
        torch = _torch()
        p = _P()
        _check(load().lbm_ade_velocity(self.ctx, ctypes.byref(p)), self.ctx)
        ts = "<f8" if self.dtype == torch.float64 else "<f4"
        return torch.as_tensor(_FieldView(p.value, (self.d, self.N), ts, self), device=self.device)

    def init(self, phi=None):
        phi_t = self._field(phi, (self.N,))
        _check(load().lbm_init(self.ctx, _ptr(phi_t), None), self.ctx)
        self._keep = (phi_t,)

    def scalar(self):
        """phi(x, t) = sum_i g_i (0 at solid cells)."""
        r = self._empty(self.N)
        _check(load().lbm_moments(self.ctx, _ptr(r), None, None), self.ctx)
        return r


# ABI-named module functions (marshalling only) -------------------------------------------------
def lbm_create(lattice, nx, ny, nz, tau, Theta, solid_mask=None, **options) -> LBM:
    return LBM(lattice, nx, ny, nz, tau, Theta, solid=solid_mask, **options)


def lbm_init(ctx: LBM, rho=None, u=None):
    ctx.init(rho, u)


def lbm_step(ctx: LBM, n: int):
    ctx.step(n)


def lbm_moments(ctx: LBM, Pi=False):
    return ctx.moments(Pi=Pi)


def lbm_totals(ctx: LBM):
    return ctx.totals()


def lbm_adjoint(ctx: LBM, loss_grad, n, checkpoint_every=0):
    ctx.adjoint(loss_grad, n, checkpoint_every)


def lbm_adjoint_release(ctx: LBM):
    ctx.adjoint_release()


def lbm_gradients(ctx: LBM):
    return ctx.gradients()


def lbm_destroy(ctx: LBM):
    ctx.close()

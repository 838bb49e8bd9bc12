"""Z-slab decomposition of a periodic box: the sharded form of the stream + collide step and of
its adjoint.

Streaming (Eq. LBE_BGK) moves every population one lattice link per time step, so a box cut
into slabs along z couples neighbouring slabs only through the populations with c_z = +-1 of
the two planes next to each cut; the adjoint's reverse streaming needs the same planes of lambda
with the opposite c_z. Each slab is a library context created with ``z_halo`` (its interior
planes plus one ghost plane below and one above); after every kernel that writes a [q][N] array
the library calls the slab's halo callback, which packs the slab's two boundary planes
(``lbm_halo_pack``), exchanges them with the neighbours, and unpacks the neighbours' planes into
the ghost planes (``lbm_halo_unpack``). Mass, momentum and the parameter gradients are sums over
cells, so a sharded run adds the slabs' FP64 values.

* :class:`HaloPlan`: which planes and directions go to which neighbour (host logic only).
* :func:`exchange`: the transport between processes, ``torch.distributed`` point-to-point
  (NCCL for device tensors, gloo for host tensors), posted in an order that pairs up even when
  both neighbours are the same rank.
* :class:`DistributedSlab`: one slab per process (rank r of R owns the r-th slab).
* :class:`SlabGroup`: several slabs of one box on one device, one host thread per slab, the
  exchange done by device copies between the slabs' buffers; the host threads meet at a barrier
  at every exchange, and no kernel ever waits for another.
"""
from __future__ import annotations

import threading

import numpy as np

from . import lbm

POP, ADJ = lbm.LBM_HALO_POPULATIONS, lbm.LBM_HALO_ADJOINT


def split(nz: int, nslabs: int):
    """(z_start, nz_local) of each slab: contiguous, sizes differing by at most one plane."""
    if nslabs < 1 or nz < nslabs:
        raise ValueError(f"cannot cut {nz} planes into {nslabs} slabs")
    base, extra = divmod(nz, nslabs)
    out, z = [], 0
    for r in range(nslabs):
        n = base + (1 if r < extra else 0)
        out.append((z, n))
        z += n
    return out


class HaloPlan:
    """Halo planes of slab `rank` of a periodic box of nz planes cut into `nslabs` slabs.

    Local plane indices count the ghost plane below as 0, so the interior is 1 .. nz_local and
    the ghost plane above is nz_local + 1. A pack on side 0 (the lowest interior plane) goes to
    the slab below, a pack on side 1 (the highest) to the slab above; the ghost plane on side 0
    receives the lower slab's side-1 pack, the one on side 1 the upper slab's side-0 pack.
    Populations stream along +c_i, so a side-0 pack carries the c_z = -1 populations and a side-1
    pack the c_z = +1 ones; lambda streams backwards and the signs flip."""

    def __init__(self, c, nz: int, nslabs: int, rank: int):
        self.c = np.asarray(c, dtype=np.int64).reshape(-1, 3)
        self.q = self.c.shape[0]
        self.nz, self.nslabs, self.rank = int(nz), int(nslabs), int(rank)
        self.parts = split(self.nz, self.nslabs)
        self.z_start, self.nz_local = self.parts[self.rank]
        self.lower = (self.rank - 1) % self.nslabs
        self.upper = (self.rank + 1) % self.nslabs

    @staticmethod
    def sign(kind: int, pack_side: int) -> int:
        return -1 if (kind == POP) == (pack_side == 0) else 1

    def pack_dirs(self, kind: int, side: int):
        s = self.sign(kind, side)
        return [i for i in range(self.q) if self.c[i, 2] == s]

    def unpack_dirs(self, kind: int, side: int):
        return self.pack_dirs(kind, 1 - side)

    def pack_plane(self, side: int) -> int:
        return 1 if side == 0 else self.nz_local

    def ghost_plane(self, side: int) -> int:
        return 0 if side == 0 else self.nz_local + 1

    def peer(self, side: int) -> int:
        """The neighbour a side-`side` pack goes to, and the one the side-`side` ghost plane
        comes from."""
        return self.lower if side == 0 else self.upper

    def global_planes(self):
        """Global z of the local planes 0 .. nz_local + 1 (periodic)."""
        return [(self.z_start - 1 + k) % self.nz for k in range(self.nz_local + 2)]

    # host reference of the library's pack / unpack on an array [q][nz_local + 2][ny][nx]
    def pack(self, kind: int, side: int, arr):
        return arr[self.pack_dirs(kind, side), self.pack_plane(side)].copy()

    def unpack(self, kind: int, side: int, arr, buf):
        arr[self.unpack_dirs(kind, side), self.ghost_plane(side)] = buf


def slab_of(field, plan: HaloPlan, nx: int, ny: int):
    """The slab's stored planes (ghosts included, taken periodically from the global field) of a
    global field [..., nz*ny*nx] (cell index x + nx (y + ny z)), flattened the same way."""
    a = np.asarray(field) if not hasattr(field, "detach") else field
    lead = tuple(a.shape[:-1])
    a3 = a.reshape(lead + (plan.nz, ny, nx))
    idx = plan.global_planes()
    out = a3[..., idx, :, :]
    return out.reshape(lead + (-1,))


def interior_of(field, plan: HaloPlan, nx: int, ny: int):
    """The interior planes of a slab field [..., (nz_local + 2)*ny*nx] as [..., nz_local, ny, nx]."""
    lead = tuple(field.shape[:-1])
    return field.reshape(lead + (plan.nz_local + 2, ny, nx))[..., 1:plan.nz_local + 1, :, :]


def exchange(plan: HaloPlan, send, recv, group=None):
    """send[side] -> neighbour plan.peer(side); recv[side] <- plan.peer(side), which sends its
    opposite side. The sends are posted side 0 then side 1 and the receives side 1 then side 0,
    so that with two slabs (lower == upper) the k-th message between the pair matches. With one
    slab the ghost planes are its own boundary planes."""
    if plan.nslabs == 1:
        recv[0].copy_(send[1])
        recv[1].copy_(send[0])
        return
    import torch.distributed as dist
    ops = [dist.P2POp(dist.isend, send[0], plan.lower, group), dist.P2POp(dist.isend, send[1], plan.upper, group),
           dist.P2POp(dist.irecv, recv[1], plan.upper, group), dist.P2POp(dist.irecv, recv[0], plan.lower, group)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()


class DistributedSlab:
    """Slab `rank` of a periodic nx*ny*nz box, one per process of a torch.distributed group;
    the halo planes travel by :func:`exchange` (NCCL between GPUs). Fields given to and returned
    by it are the slab's own stored planes (:func:`slab_of` / :func:`interior_of`)."""

    def __init__(self, lattice, nx, ny, nz, tau, Theta, solid=None, group=None, **kw):
        import torch
        import torch.distributed as dist
        self.group = group
        world = dist.get_world_size(group) if dist.is_initialized() else 1
        rank = dist.get_rank(group) if dist.is_initialized() else 0
        c, _ = lbm.lattice_info(int(lattice))
        self.plan = HaloPlan(c, nz, world, rank)
        self.nx, self.ny = int(nx), int(ny)
        mask = None if solid is None else slab_of(np.asarray(solid, np.uint8), self.plan, nx, ny)
        self.L = lbm.LBM(lattice, nx, ny, self.plan.nz_local, tau, Theta, solid=mask, z_halo=True,
                         halo=self._halo, **kw)
        dev = self.L.device
        self.send = [[torch.empty(self.L.halo_bytes(k), dtype=torch.uint8, device=dev) for _ in (0, 1)] for k in (0, 1)]
        self.recv = [[torch.empty(self.L.halo_bytes(k), dtype=torch.uint8, device=dev) for _ in (0, 1)] for k in (0, 1)]

    def _halo(self, kind, array):
        L = self.L
        L.halo_pack(kind, 0, array, self.send[kind][0])
        L.halo_pack(kind, 1, array, self.send[kind][1])
        exchange(self.plan, self.send[kind], self.recv[kind], self.group)
        L.halo_unpack(kind, 0, array, self.recv[kind][0])
        L.halo_unpack(kind, 1, array, self.recv[kind][1])

    def _sum(self, values):
        import torch
        import torch.distributed as dist
        t = torch.tensor(values, dtype=torch.float64, device=self.L.device)
        if self.plan.nslabs > 1:
            dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def totals(self):
        m, p = self.L.totals()
        s = self._sum([m, *p])
        return float(s[0]), s[1:]

    def gradients(self, du0=True):
        dth, dtau, g = self.L.gradients(du0=du0)
        s = self._sum([*dth, dtau])
        return s[:-1], float(s[-1]), g


class SlabGroup:
    """A periodic nx*ny*nz box cut into `nslabs` z-slabs that all live on one device, with the
    library's calls of the whole box: init / step / moments / populations / totals /
    record_checkpoints / adjoint / gradients on global fields. Each slab has its own stream and
    host thread; at every exchange a slab packs its boundary planes, waits at a barrier until
    all slabs have packed, unpacks its neighbours' planes after their pack events, and waits at a
    second barrier before going on (so no pack buffer is overwritten while a neighbour reads it).
    Host threads wait on each other, kernels never do."""

    def __init__(self, lattice, nx, ny, nz, tau, Theta, nslabs, solid=None, timeout=300.0, **kw):
        import torch
        self.q, self.nx, self.ny, self.nz = int(lattice), int(nx), int(ny), int(nz)
        self.d = lbm.D_OF_Q[self.q]
        c, _ = lbm.lattice_info(self.q)
        self.plans = [HaloPlan(c, nz, nslabs, r) for r in range(nslabs)]
        self.nslabs = int(nslabs)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(nslabs)]
        self.events = [torch.cuda.Event() for _ in range(nslabs)]
        self.barrier = threading.Barrier(nslabs, timeout=timeout)
        self.kinds = [None] * nslabs
        self.exchanges = 0
        self.ctx = []
        for r, plan in enumerate(self.plans):
            mask = None if solid is None else slab_of(np.asarray(solid, np.uint8), plan, nx, ny)
            L = lbm.LBM(lattice, nx, ny, plan.nz_local, tau, Theta, solid=mask, stream=self.streams[r],
                        z_halo=True, halo=self._make_halo(r), **kw)
            self.ctx.append(L)
        self.send = [[[torch.empty(L.halo_bytes(k), dtype=torch.uint8, device=self.device) for _ in (0, 1)]
                      for k in (0, 1)] for L in self.ctx]
        self.dtype = self.ctx[0].dtype

    # -- exchange ---------------------------------------------------------------------------------
    def _make_halo(self, r):
        def halo(kind, array):
            L, s, plan = self.ctx[r], self.streams[r], self.plans[r]
            L.halo_pack(kind, 0, array, self.send[r][kind][0])
            L.halo_pack(kind, 1, array, self.send[r][kind][1])
            self.events[r].record(s)
            self.kinds[r] = kind
            self.barrier.wait()
            if any(k != kind for k in self.kinds):
                raise RuntimeError("z-slabs out of step: exchange kinds %s" % self.kinds)
            s.wait_event(self.events[plan.lower])
            s.wait_event(self.events[plan.upper])
            L.halo_unpack(kind, 0, array, self.send[plan.lower][kind][1])
            L.halo_unpack(kind, 1, array, self.send[plan.upper][kind][0])
            s.synchronize()
            if r == 0:
                self.exchanges += 1
            self.barrier.wait()
        return halo

    def _run(self, fn):
        """fn(r, ctx) in one thread per slab with the slab's stream current; re-raises the first
        failure (the other threads leave at the broken barrier)."""
        import torch
        errs = [None] * self.nslabs

        def work(r):
            try:
                with torch.cuda.device(self.device), torch.cuda.stream(self.streams[r]):
                    fn(r, self.ctx[r])
            except BaseException as e:  # noqa: BLE001 - reported below
                errs[r] = e
                self.barrier.abort()

        th = [threading.Thread(target=work, args=(r,)) for r in range(self.nslabs)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for s in self.streams:
            s.synchronize()
        if any(e is not None for e in errs):
            self.barrier.reset()
            first = next((e for e in errs if e is not None and not isinstance(e, threading.BrokenBarrierError)),
                         next(e for e in errs if e is not None))
            raise first

    # -- fields -------------------------------------------------------------------------------------
    def _slab_fields(self, x, r):
        import torch
        if x is None:
            return None
        t = x if isinstance(x, torch.Tensor) else torch.as_tensor(np.asarray(x))
        t = t.to(device=self.device, dtype=self.dtype)
        return slab_of(t, self.plans[r], self.nx, self.ny).contiguous()

    def _gather(self, parts):
        import torch
        inner = [interior_of(p, self.plans[r], self.nx, self.ny) for r, p in enumerate(parts)]
        return torch.cat(inner, dim=-3).reshape(inner[0].shape[:-3] + (-1,))

    # -- the box's calls --------------------------------------------------------------------------
    def init(self, rho=None, u=None):
        fr = [self._slab_fields(rho, r) for r in range(self.nslabs)]
        fu = [None if u is None else self._slab_fields(
            (u if hasattr(u, "reshape") else np.asarray(u)).reshape(self.d, -1), r) for r in range(self.nslabs)]
        self._keep = (fr, fu)
        self._run(lambda r, L: L.init(fr[r], fu[r]))

    def step(self, n=1):
        self._run(lambda r, L: L.step(n))

    def record_checkpoints(self, k):
        for L in self.ctx:
            L.record_checkpoints(k)

    def moments(self, Pi=False):
        outs = [None] * self.nslabs

        def m(r, L):
            outs[r] = L.moments(Pi=Pi)
            L.sync()
        self._run(m)
        rho = self._gather([o[0] for o in outs])
        u = self._gather([o[1] for o in outs])
        P = self._gather([o[2] for o in outs]) if Pi else None
        return rho, u, P

    def populations(self):
        outs = [None] * self.nslabs

        def p(r, L):
            outs[r] = L.populations()
            L.sync()
        self._run(p)
        return self._gather(outs)

    def totals(self):
        m, p = 0.0, np.zeros(self.d)
        for L in self.ctx:
            mm, pp = L.totals()
            m += mm
            p += pp
        return m, p

    def adjoint(self, loss_grad, n, checkpoint_every=0):
        g = [self._slab_fields(loss_grad.reshape(self.d, -1), r) for r in range(self.nslabs)]
        self._run(lambda r, L: L.adjoint(g[r], n, checkpoint_every))

    def gradients(self):
        dth, dtau, du0 = 0.0, 0.0, []
        for L in self.ctx:
            a, b, c = L.gradients()
            dth = dth + a
            dtau += b
            du0.append(c)
        return dth, dtau, self._gather(du0)

    @property
    def launches(self):
        return sum(L.launches for L in self.ctx)

    def close(self):
        for L in self.ctx:
            L.close()

"""Host logic of the z-slab decomposition (no GPU): the halo plan against brute-force streaming
on a global array, and the torch.distributed exchange with world size 2 and 3 over gloo.

Streaming of Eq. LBE_BGK gathers f_i(x) = f*_i(x - c_i) from post-collision populations; the
adjoint's reverse streaming gathers mu_i(x) = lambda_i(x + c_i). A slab must see, after the
exchange, exactly what the whole periodic box would give at every interior cell."""
import socket

import numpy as np
import pytest

from paper_2605_27004_gb300 import slabs

POP, ADJ = slabs.POP, slabs.ADJ


def _velocities(q):
    """The library's direction order (opposite pairs 2k+1, 2k+2 after the rest velocity), built
    here from the half-vectors so the test needs neither the library nor a GPU."""
    half = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1),
            (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)]
    n = 9 if q == 19 else 13
    c = [(0, 0, 0)]
    for v in half[:n]:
        c += [v, tuple(-a for a in v)]
    return np.array(c)


def _gather(arr, c, sign):
    """out_i(x) = arr_i(x - sign * c_i) on a periodic [q][nz][ny][nx] array."""
    out = np.empty_like(arr)
    for i, (cx, cy, cz) in enumerate(c):
        out[i] = np.roll(arr[i], (sign * cz, sign * cy, sign * cx), axis=(0, 1, 2))
    return out


def test_split_is_contiguous_and_balanced():
    for nz, s in [(10, 3), (7, 7), (64, 4), (5, 2)]:
        parts = slabs.split(nz, s)
        assert parts[0][0] == 0
        assert sum(n for _, n in parts) == nz
        assert all(parts[k][0] + parts[k][1] == parts[k + 1][0] for k in range(s - 1))
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        slabs.split(3, 4)


@pytest.mark.parametrize("q,ndir", [(19, 5), (27, 9)])
def test_plan_directions(q, ndir):
    c = _velocities(q)
    p = slabs.HaloPlan(c, 8, 2, 0)
    for kind in (POP, ADJ):
        for side in (0, 1):
            dirs = p.pack_dirs(kind, side)
            assert len(dirs) == ndir
            want = (-1 if side == 0 else 1) * (1 if kind == POP else -1)
            assert all(c[i, 2] == want for i in dirs)
            assert p.unpack_dirs(kind, side) == p.pack_dirs(kind, 1 - side)


def _exchange_local(arrs, plans, kind):
    """All slabs of one process: pack, then unpack the neighbours' packs."""
    packs = [[p.pack(kind, s, a) for s in (0, 1)] for p, a in zip(plans, arrs)]
    for p, a in zip(plans, arrs):
        p.unpack(kind, 0, a, packs[p.lower][1])
        p.unpack(kind, 1, a, packs[p.upper][0])


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("nz,nslabs", [(9, 1), (9, 2), (10, 3), (6, 6)])
@pytest.mark.parametrize("kind", [POP, ADJ])
def test_exchange_gives_the_whole_box_streaming(q, nz, nslabs, kind):
    """After the exchange every interior cell of every slab gathers what the periodic box gives:
    populations by the pull rule f_i(x) = f*_i(x - c_i), lambda by mu_i(x) = lambda_i(x + c_i)."""
    rng = np.random.default_rng(10 * q + nz + nslabs)
    c = _velocities(q)
    nx, ny = 5, 4
    A = rng.standard_normal((q, nz, ny, nx))
    sign = 1 if kind == POP else -1
    want = _gather(A, c, sign)
    plans = [slabs.HaloPlan(c, nz, nslabs, r) for r in range(nslabs)]
    arrs = []
    for p in plans:
        a = slabs.slab_of(A.reshape(q, -1), p, nx, ny).reshape(q, p.nz_local + 2, ny, nx).copy()
        a[:, 0] = np.nan  # ghost planes start unknown
        a[:, -1] = np.nan
        arrs.append(a)
    _exchange_local(arrs, plans, kind)
    for p, a in zip(plans, arrs):
        # gather on the slab: z never wraps for interior cells, x and y wrap periodically
        got = np.empty((q, p.nz_local, ny, nx))
        for i, (cx, cy, cz) in enumerate(c):
            zsrc = np.arange(1, p.nz_local + 1) - sign * cz
            got[i] = np.roll(a[i][zsrc], (sign * cy, sign * cx), axis=(1, 2))
        ref = want[:, p.z_start:p.z_start + p.nz_local]
        assert np.array_equal(got, ref)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _dist_worker(rank, world, port, q, nz, kind, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = _velocities(q)
        nx, ny = 4, 3
        A = np.random.default_rng(5).standard_normal((q, nz, ny, nx))
        p = slabs.HaloPlan(c, nz, world, rank)
        a = slabs.slab_of(A.reshape(q, -1), p, nx, ny).reshape(q, p.nz_local + 2, ny, nx).copy()
        a[:, 0] = np.nan
        a[:, -1] = np.nan
        send = [torch.as_tensor(p.pack(kind, s, a)).contiguous() for s in (0, 1)]
        recv = [torch.empty_like(send[s]) for s in (0, 1)]
        slabs.exchange(p, send, recv)
        p.unpack(kind, 0, a, recv[0].numpy())
        p.unpack(kind, 1, a, recv[1].numpy())
        planes = p.global_planes()
        ok = True
        for side in (0, 1):
            g = p.ghost_plane(side)
            dirs = p.unpack_dirs(kind, side)
            ok &= np.array_equal(a[dirs, g], A[dirs, planes[g]])
        out[rank] = int(ok)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nz", [(2, 6), (3, 7)])
@pytest.mark.parametrize("kind", [POP, ADJ])
def test_distributed_exchange_gloo(world, nz, kind):
    """torch.distributed point-to-point exchange between ranks (gloo on the CPU): each rank's
    ghost planes hold its neighbours' boundary planes of the global array, also with two ranks,
    where both neighbours are the same process."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_dist_worker, args=(r, world, port, 19, nz, kind, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {r: 1 for r in range(world)}


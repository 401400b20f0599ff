"""Y-slab decomposition of one grid (paper_2606_02711_gb300/slabs.py) on CPU
ranks with gloo, the oracle advancing each rank's slab: with the halo rows
swapped before every substep and the global time step, the rows each rank
owns equal the single-domain oracle run bit for bit (Cartesian with outflow
edges, axisymmetric with the midplane mirror and vacuum outer edge)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_02711_gb300 import slabs

NSTEPS = 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cloud(geometry):
    import workloads as wl
    c = wl.lognormal_cloud(20, 17, seed=191, v_edge_kms=150.0, Z=0.3, p_d=1e-7)
    c.geometry = geometry
    c.bc = (0, 1, 0, 1) if geometry == 1 else (1, 1, 1, 1)
    return c


def _state(c):
    g = np.random.default_rng(192)
    J = 1e-3 * np.exp(g.normal(0, 0.5, (194, c.ny, c.nx)))
    return J, 0.4 * J * g.uniform(-1, 1, J.shape), 0.4 * J * g.uniform(-1, 1, J.shape)


def _slab_oracle(c, e0, e1, ny):
    import oracle
    kw = c.kwargs()
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        kw[f] = np.ascontiguousarray(np.broadcast_to(kw[f], (ny, c.nx))[e0:e1])
    kw["ny"] = e1 - e0
    bc = list(kw["bc"])
    if e0 > 0:
        bc[2] = 0  # interior edges: whatever ghosts, only the halo rows see them
    if e1 < ny:
        bc[3] = 0
    kw["bc"] = tuple(bc)
    return oracle.Oracle(edges=oracle.freq_grid(), **kw)


def _worker(rank, world, port, geometry, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    oracle.set_threads(1)  # one thread per rank: the ranks share the host's cores
    c = _cloud(geometry)
    ny = c.ny
    slabs.check_split(ny, world)
    y0, y1 = slabs.slab_rows(ny, world, rank)
    e0, e1 = slabs.extended_rows(ny, world, rank)
    O = _slab_oracle(c, e0, e1, ny)
    dt = slabs.global_dt(O.dt_cfl)
    J, Hx, Hy = (np.ascontiguousarray(a[:, e0:e1]) for a in _state(c))
    fx = fy = None
    for _ in range(NSTEPS):
        slabs.exchange((J, Hx, Hy), ny, world, rank)
        J, Hx, Hy, fx, fy, _ = O.substep(J, Hx, Hy, dt)
    own = slice(y0 - e0, y1 - e0)
    mine = (y0, y1, J[:, own], Hx[:, own], Hy[:, own], fx[own], fy[own], dt)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _worker_ctilde(rank, world, port, geometry, out):
    # two dynamic c_tilde updates from 1e8 cm/s (the first bound by the x4
    # rate limit), each followed by two substeps
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    oracle.set_threads(1)  # one thread per rank: the ranks share the host's cores
    c = _cloud(geometry)
    ny = c.ny
    y0, y1 = slabs.slab_rows(ny, world, rank)
    e0, e1 = slabs.extended_rows(ny, world, rank)
    O = _slab_oracle(c, e0, e1, ny)
    O.set_ctilde(1e8)
    J, Hx, Hy = (np.ascontiguousarray(a[:, e0:e1]) for a in _state(c))
    cts = []
    for _ in range(2):
        ct = slabs.global_ctilde(O.dynamic_ctilde())
        O.set_ctilde(ct)
        cts.append(ct)
        dt = slabs.global_dt(O.dt_cfl)
        for _ in range(2):
            slabs.exchange((J, Hx, Hy), ny, world, rank)
            J, Hx, Hy, _, _, _ = O.substep(J, Hx, Hy, dt)
    own = slice(y0 - e0, y1 - e0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (y0, y1, J[:, own], cts))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _run_workers(target, world, geometry):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, geometry, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return gathered


def _worker_rows(rank, world, port, ny, out):
    # each rank fills its own rows with their global row index (halo rows -1),
    # as a numpy array and as a torch tensor, and swaps the halos
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y0, y1 = slabs.slab_rows(ny, world, rank)
    e0, e1 = slabs.extended_rows(ny, world, rank)
    rows = np.arange(e0, e1, dtype=np.float64)
    a = np.where((rows >= y0) & (rows < y1), rows, -1.0)[None, :, None] * np.ones((3, 1, 5))
    t = torch.from_numpy(a.copy())
    slabs.exchange((a, t), ny, world, rank)
    out.put((rank, a, t.numpy(), rows))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ny,world", [(9, 4), (17, 3), (4, 2)])
def test_exchange_fills_every_halo_row_from_its_owner(ny, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_rows, args=(r, world, port, ny, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, a, t, rows in res:
        want = np.broadcast_to(rows[None, :, None], a.shape)
        np.testing.assert_array_equal(a, want)
        np.testing.assert_array_equal(t, want)


class _RowCtx:
    """A stand-in for a slab context's row calls (lym1_get_rows /
    lym1_set_rows) over numpy state arrays of one element type."""

    def __init__(self, arrays):
        self.a = arrays
        self.nb, _, self.nx = arrays[0].shape

    def state_itemsize(self):
        return self.a[0].dtype.itemsize

    def get_rows(self, y0, n, out):
        import torch
        for o, a in zip(out, self.a):
            o.copy_(torch.from_numpy(np.ascontiguousarray(a[:, y0:y0 + n])))
        return out

    def set_rows(self, y0, J, Hx, Hy):
        for a, t in zip(self.a, (J, Hx, Hy)):
            a[:, y0:y0 + t.shape[1]] = t.numpy()


def _worker_ctx_rows(rank, world, port, ny, out):
    # the row-call exchange in both element types: each rank's own rows hold
    # their global row index (halo rows -1) before the swap
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y0, y1 = slabs.slab_rows(ny, world, rank)
    e0, e1 = slabs.extended_rows(ny, world, rank)
    rows = np.arange(e0, e1, dtype=np.float64)
    res = []
    for dt in (np.float32, np.float64):
        a = [(np.where((rows >= y0) & (rows < y1), rows, -1.0)[None, :, None] * np.ones((3, 1, 5)) *
              (i + 1)).astype(dt) for i in range(3)]
        slabs.exchange_ctx(_RowCtx(a), ny, world, rank)
        res.append(a)
    out.put((rank, res, rows))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ny,world", [(9, 4), (17, 3), (4, 2)])
def test_row_call_exchange_fills_every_halo_row_from_its_owner(ny, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_ctx_rows, args=(r, world, port, ny, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, per_type, rows in res:
        for a in per_type:
            for i, arr in enumerate(a):
                want = np.broadcast_to(rows[None, :, None] * (i + 1), arr.shape).astype(arr.dtype)
                np.testing.assert_array_equal(arr, want)


def test_split_is_a_balanced_partition():
    for ny in (4, 17, 512, 2048):
        for world in (1, 2, 3, 8):
            if ny < 2 * world:
                continue
            rows = [slabs.slab_rows(ny, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [y1 - y0 for y0, y1 in rows]
            assert max(sizes) - min(sizes) <= 1
            slabs.check_split(ny, world)
    with pytest.raises(ValueError):
        slabs.check_split(5, 3)


@pytest.mark.parametrize("geometry,world", [(0, 2), (0, 3), (1, 3)])
def test_decomposed_run_equals_single_domain(geometry, world):
    import oracle
    c = _cloud(geometry)
    ref_O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    (J, Hx, Hy, fx, fy), _ = ref_O.run(NSTEPS, _state(c))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, geometry, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for y0, y1, Js, Hxs, Hys, fxs, fys, dt in gathered:
        assert dt == ref_O.dt_cfl
        np.testing.assert_array_equal(Js, J[:, y0:y1])
        np.testing.assert_array_equal(Hxs, Hx[:, y0:y1])
        np.testing.assert_array_equal(Hys, Hy[:, y0:y1])
        np.testing.assert_array_equal(fxs, fx[y0:y1])
        np.testing.assert_array_equal(fys, fy[y0:y1])


@pytest.mark.parametrize("geometry,world", [(0, 3), (1, 2)])
def test_decomposed_dynamic_ctilde_equals_single_domain(geometry, world):
    import oracle
    c = _cloud(geometry)
    ref_O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    ref_O.set_ctilde(1e8)
    st = _state(c)
    cts = []
    for _ in range(2):
        cts.append(ref_O.dynamic_ctilde())
        st, _ = ref_O.run(2, st)
        st = st[:3]
    assert cts[0] == 4e8 and cts[1] > cts[0]  # rate-limited, then the rule's own value
    # the deciding cell sits in one slab: the others reach lower values
    local = []
    for r in range(world):
        e0, e1 = slabs.extended_rows(c.ny, world, r)
        O = _slab_oracle(c, e0, e1, c.ny)
        O.set_ctilde(4e8)
        local.append(O.dynamic_ctilde())
    assert max(local) == cts[1] and min(local) < cts[1]
    for y0, y1, Js, got in _run_workers(_worker_ctilde, world, geometry):
        assert got == cts
        np.testing.assert_array_equal(Js, st[0][:, y0:y1])

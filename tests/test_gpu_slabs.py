"""Halo rows of the y-slab split on the GPU (lym1_get_rows / lym1_set_rows):
the row calls agree with the whole-state calls in the state's own element
type, and two slab contexts on one GPU whose two edge rows are swapped through
them before every substep reproduce the single-domain run in their own rows
(bit for bit under LYM1_FP64_DET; under LYM1_MIXED the state bit for bit and
the force to its summation order).  The exchange here copies between the two
contexts directly; paper_2606_02711_gb300.slabs.exchange_ctx moves the same
rows between ranks (tested with gloo in test_slabs.py)."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from paper_2606_02711_gb300 import slabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


def _cloud(geometry=0):
    c = wl.lognormal_cloud(24, 21, seed=301, v_edge_kms=150.0, Z=0.3, p_d=1e-7)
    c.geometry = geometry
    c.bc = (0, 1, 0, 1) if geometry == 1 else (1, 1, 1, 1)
    return c


def _slab_cloud(c, e0, e1):
    """The cloud's rows [e0, e1); interior edges take zero-gradient ghosts,
    which only the halo rows see."""
    f = {}
    for name in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        f[name] = np.ascontiguousarray(np.broadcast_to(getattr(c, name), (c.ny, c.nx))[e0:e1])
    bc = list(c.bc)
    if e0 > 0:
        bc[2] = 0
    if e1 < c.ny:
        bc[3] = 0
    return dataclasses.replace(c, ny=e1 - e0, bc=tuple(bc), **f)


@pytest.mark.parametrize("precision", [0, 2])
def test_rows_agree_with_the_whole_state(L, precision):
    torch = pytest.importorskip("torch")
    c = _cloud()
    ctx = L.from_cloud(c, precision=precision)
    st = wl.populated_state(c, ctx.nb, seed=302)
    ctx.set_state(*st)
    J, Hx, Hy = ctx.get_state()
    dt = np.float32 if ctx.state_itemsize() == 4 else np.float64
    assert ctx.state_itemsize() == (4 if precision >= 2 else 8)
    # host buffers: rows 5..8 out, equal to the state rounded to the element type
    rows = ctx.get_rows(5, 4)
    for a, ref in zip(rows, (J, Hx, Hy)):
        assert a.dtype == dt and a.shape == (ctx.nb, 4, c.nx)
        np.testing.assert_array_equal(a.astype(np.float64), ref[:, 5:9])
    # device buffers: write rows 0..2 with rows 10..12 and read the whole state back
    src = ctx.get_rows(10, 3, tuple(torch.empty((ctx.nb, 3, c.nx), dtype=torch.from_numpy(
        np.zeros(1, dt)).dtype, device="cuda") for _ in range(3)))
    ctx.set_rows(0, *src)
    J2, Hx2, Hy2 = ctx.get_state()
    for a, ref in zip((J2, Hx2, Hy2), (J, Hx, Hy)):
        np.testing.assert_array_equal(a[:, 0:3], ref[:, 10:13])
        np.testing.assert_array_equal(a[:, 3:], ref[:, 3:])
    # the whole grid, and nothing at all
    full = ctx.get_rows(0, c.ny)
    np.testing.assert_array_equal(full[0].astype(np.float64), J2)
    ctx.set_rows(0, *(np.empty((ctx.nb, 0, c.nx), dtype=dt) for _ in range(3)))
    # rows outside the grid, a wrong element type
    with pytest.raises(L.Lym1Error):
        ctx.get_rows(c.ny - 2, 3)
    with pytest.raises(L.Lym1Error):
        ctx.get_rows(-1, 2)
    with pytest.raises(TypeError):
        ctx.set_rows(0, *(np.zeros((ctx.nb, 1, c.nx), dtype=np.float16) for _ in range(3)))
    ctx.destroy()


def _swap_halos(ctxs, ny, world):
    """exchange_ctx's row moves between contexts on one GPU: every rank's
    HALO lowest and highest own rows into its neighbours' halo rows."""
    moves = []
    for r in range(world):
        y0, y1 = slabs.slab_rows(ny, world, r)
        e0, _ = slabs.extended_rows(ny, world, r)
        if r > 0:  # own lowest rows -> the upper halo of rank r - 1
            pe0, _ = slabs.extended_rows(ny, world, r - 1)
            moves.append((r, y0 - e0, r - 1, y0 - pe0))
        if r < world - 1:  # own highest rows -> the lower halo of rank r + 1
            ne0, _ = slabs.extended_rows(ny, world, r + 1)
            moves.append((r, y1 - slabs.HALO - e0, r + 1, y1 - slabs.HALO - ne0))
    rows = [ctxs[a].get_rows(ra, slabs.HALO) for a, ra, _, _ in moves]
    for (_, _, b, rb), (J, Hx, Hy) in zip(moves, rows):
        ctxs[b].set_rows(rb, J, Hx, Hy)


@pytest.mark.parametrize("precision,geometry,world", [(0, 0, 2), (0, 1, 3), (2, 0, 3)])
def test_slabs_on_one_gpu_equal_the_single_domain(L, precision, geometry, world):
    c = _cloud(geometry)
    ny, nsteps = c.ny, 4
    ref = L.from_cloud(c, precision=precision)
    st = wl.populated_state(c, ref.nb, seed=303)
    ref.set_state(*st)
    ctxs, spans = [], []
    for r in range(world):
        e0, e1 = slabs.extended_rows(ny, world, r)
        x = L.from_cloud(_slab_cloud(c, e0, e1), precision=precision)
        x.set_state(*(np.ascontiguousarray(a[:, e0:e1]) for a in st))
        ctxs.append(x)
        spans.append((e0, e1))
    dt = min(x.dt_cfl for x in ctxs)
    assert dt >= ref.dt_cfl
    for _ in range(nsteps):
        _swap_halos(ctxs, ny, world)
        for x in ctxs:
            x.substeps(1, dt)
        ref.substeps(1, dt)
    J, Hx, Hy = ref.get_state()
    fx, fy = ref.force()
    for r, (x, (e0, e1)) in enumerate(zip(ctxs, spans)):
        y0, y1 = slabs.slab_rows(ny, world, r)
        own = slice(y0 - e0, y1 - e0)
        Js, Hxs, Hys = x.get_state()
        fxs, fys = x.force()
        for a, b in ((Js, J), (Hxs, Hx), (Hys, Hy)):
            np.testing.assert_array_equal(a[:, own], b[:, y0:y1])
        for a, b in ((fxs, fx), (fys, fy)):
            if precision == 0:
                np.testing.assert_array_equal(a[own], b[y0:y1])
            else:
                np.testing.assert_allclose(a[own], b[y0:y1], rtol=1e-12,
                                           atol=1e-12 * np.abs(b).max())
        x.destroy()
    ref.destroy()

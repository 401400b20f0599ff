"""Work layouts of the batched transport (tile shape 16 x 16 or 32 x 8, and the
bins of each tile split over 1, 2, 4 or 8 blocks) and their autotuner.

A layout changes which block computes which (cell, bin), not what is
computed, so J and H are bit for bit the same under every layout; the force
of a split tile is the sum of its groups' sums (added in group order), and the
transport's bookkeeping is summed over other blocks, so those change only in
their rounding.  Under LYM1_FP64_DET every layout gives the oracle's state bit
for bit, and the force too with unsplit tiles.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

LAYOUTS = [(0, 1), (1, 1), (0, 2), (0, 4), (0, 8)]


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.mark.parametrize("shape,groups", LAYOUTS)
def test_every_layout_gives_the_oracle_state_under_fp64_det(L, shape, groups):
    c = wl.lognormal_cloud(45, 38, seed=3, v_edge_kms=30.0)
    st = wl.populated_state(c, 194, seed=4)
    edges = oracle.freq_grid()
    ctx = L.from_cloud(c, precision=L.FP64_DET, edges=edges)
    ctx.set_state(*st)
    b = L.Batch([ctx])
    b.configure(shape, groups, 0)
    cfg = b.config()
    assert (cfg["tile_x"], cfg["tile_y"], cfg["bin_groups"]) == (
        (16, 16) if shape == 0 else (32, 8)) + (groups,)
    b.substeps(3)
    b.destroy()
    got = ctx.get_state() + ctx.force()
    dg = ctx.diagnostics()
    ctx.destroy()
    ref, diags = oracle.Oracle(edges=edges, **c.kwargs()).run(3, st)
    for a, r, n in zip(got[:3], ref[:3], ("J", "Hx", "Hy")):
        assert np.array_equal(a, r), n
    for a, r, n in zip(got[3:], ref[3:], ("fx", "fy")):
        if groups == 1:
            assert np.array_equal(a, r), n
        else:  # the groups' sums added in group order: rounding only
            np.testing.assert_allclose(a, r, rtol=1e-13, atol=1e-13 * np.abs(r).max(), err_msg=n)
    for k in ("emitted", "absorbed", "outflow", "work"):
        assert dg[k] == pytest.approx(sum(x[k] for x in diags), rel=1e-12), k
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fast"])
def test_layouts_agree_under_the_tuned_policies(L, precision):
    # a face on a tile's edge is evaluated by the edge threads of one tile and
    # by the regular face code of the next: both must round alike
    c = wl.lognormal_cloud(48, 40, seed=5, L_sun=1e7)
    st = wl.populated_state(c, 194, seed=6)
    out = []
    for shape, groups in LAYOUTS:
        ctx = L.from_cloud(c, precision=precision)
        ctx.set_state(*st)
        b = L.Batch([ctx])
        b.configure(shape, groups, 0)
        b.substeps(4)
        b.destroy()
        out.append(ctx.get_state() + ctx.force())
        ctx.destroy()
    ftol = 1e-12 if precision != "mixed_fast" else 1e-5  # FP32 per-cell force sums
    for lay, got in zip(LAYOUTS[1:], out[1:]):
        for a, r, n in zip(got[:3], out[0][:3], ("J", "Hx", "Hy")):
            assert np.array_equal(a, r), (lay, n, int(np.sum(a != r)))
        for a, r, n in zip(got[3:], out[0][3:], ("fx", "fy")):
            np.testing.assert_allclose(a, r, rtol=ftol, atol=ftol * np.abs(r).max(),
                                       err_msg=f"{lay} {n}")


def test_tuner_chooses_and_caches_a_layout(L):
    clouds = [wl.lognormal_cloud(32, 32, seed=41), wl.lognormal_cloud(48, 32, seed=42),
              wl.lognormal_cloud(40, 24, seed=43)]
    ctxs = [L.from_cloud(c, precision=L.MIXED_FAST) for c in clouds]
    b = L.Batch(ctxs)
    b.substeps(40)  # more than the candidates: tuning, then graph replay
    cfg = b.config()
    b.destroy()
    assert (cfg["tile_x"], cfg["tile_y"]) in ((16, 16), (32, 8))
    assert cfg["bin_groups"] in (1, 2, 4, 8) and cfg["grid_t"] > 0 and cfg["grid_f"] > 0
    # small clouds: a few dozen tiles do not fill 152 SMs, so split tiles were candidates
    b2 = L.Batch(ctxs)  # same class: tuned at creation from the cache
    assert b2.config() == cfg
    b2.destroy()
    for ctx in ctxs:
        ctx.destroy()


def test_configure_refuses_invalid_layouts(L):
    c = wl.lognormal_cloud(16, 16, seed=5)
    ctx = L.from_cloud(c, precision=L.MIXED)
    ctx.set_pruning(1e-10)
    b = L.Batch([ctx])
    with pytest.raises(L.Lym1Error):
        b.configure(1, 1, 0)  # 32 x 8 tiles only in the plain table modes
    for bad in ((2, 1, 0), (0, 3, 0), (0, 16, 0), (0, 1, -1)):
        with pytest.raises(L.Lym1Error):
            b.configure(*bad)
    b.configure(0, 2, 0)
    b.substeps(1)
    b.destroy()
    ctx.destroy()

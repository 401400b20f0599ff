"""Batched substeps (one persistent launch per kernel over several clouds,
CUDA-graph replay, tuned persistent grid) give every cloud exactly the result
it gets alone."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


def _clouds():
    return [wl.lognormal_cloud(40, 24, seed=21, mean_nh=3e2, L_sun=1e5, Z=0.0),
            wl.lognormal_cloud(96, 80, seed=22, mean_nh=1e4, L_sun=1e7, Z=1e-2),
            wl.lognormal_cloud(17, 33, seed=23, mean_nh=1e3, L_sun=1e6, Z=1e-3)]


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batch_equals_individual_runs(L, precision):
    edges = oracle.freq_grid()
    clouds = _clouds()
    solo = []
    for c in clouds:
        ctx = L.from_cloud(c, precision=precision, edges=edges)
        ctx.substeps(9)
        solo.append(ctx.get_state() + ctx.force() + (ctx.diagnostics(),))
        ctx.destroy()
    ctxs = [L.from_cloud(c, precision=precision, edges=edges) for c in clouds]
    b = L.Batch(ctxs)
    b.substeps(5)   # tuning substeps, then graph replay
    b.substeps(4)
    gt, gf = b.grid()
    assert gt > 0 and gf > 0
    b.destroy()
    for ctx, ref in zip(ctxs, solo):
        got = ctx.get_state() + ctx.force()
        for a, r in zip(got, ref[:5]):
            assert np.array_equal(a, r)
        d = ctx.diagnostics()
        for k in ("e_tot", "emitted", "absorbed", "outflow", "work", "substeps"):
            assert d[k] == ref[5][k], k
        ctx.destroy()


def test_batch_rejects_mixed_precisions(L):
    c = wl.lognormal_cloud(16, 16, seed=3)
    a = L.from_cloud(c, precision=0)
    b = L.from_cloud(c, precision=3)
    with pytest.raises(L.Lym1Error):
        L.Batch([a, b])
    a.destroy()
    b.destroy()

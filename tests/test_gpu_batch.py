"""Batched substeps (one persistent launch per kernel over several clouds,
CUDA-graph replay, tuned persistent grid and transport layout) give every
cloud the result it gets alone: bit for bit under LYM1_FP64_DET, whose batches
keep one 16 x 16 block per tile.  Under the other policies the tuner may pick
another layout for a batch than for a cloud alone; J and H are still the same
bit for bit, and the force and the transport's bookkeeping differ only in
their summation order (FP64 sums: 1e-12; FP32 per-cell sums of
LYM1_MIXED_FAST: 1e-6)."""
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
    rel = 0.0 if precision == 0 else (1e-6 if precision == 3 else 1e-12)
    for ctx, ref in zip(ctxs, solo):
        got = ctx.get_state() + ctx.force()
        for a, r in zip(got[:3], ref[:3]):
            assert np.array_equal(a, r)
        for a, r in zip(got[3:], ref[3:5]):
            if rel == 0.0:
                assert np.array_equal(a, r)
            else:
                np.testing.assert_allclose(a, r, rtol=rel, atol=rel * np.abs(r).max())
        d = ctx.diagnostics()
        assert d["e_tot"] == ref[5]["e_tot"] and d["substeps"] == ref[5]["substeps"]
        for k in ("emitted", "absorbed", "outflow", "work"):
            assert d[k] == pytest.approx(ref[5][k], rel=rel, abs=0.0), k
        ctx.destroy()


def test_batch_rejects_mixed_precisions(L):
    c = wl.lognormal_cloud(16, 16, seed=3)
    a = L.from_cloud(c, precision=0)
    b = L.from_cloud(c, precision=3)
    with pytest.raises(L.Lym1Error):
        L.Batch([a, b])
    a.destroy()
    b.destroy()

"""Checkpoint/resume and the failure path of the kernels' bounded waits."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 3])
def test_resume_equals_uninterrupted_run(precision):
    import paper_2606_02711_gb300.lym1 as L
    c = wl.lognormal_cloud(48, 40, seed=41, v_edge_kms=50.0)
    a = L.from_cloud(c, precision=precision)
    a.substeps(7)
    ref = a.get_state() + a.force()
    a.destroy()
    b = L.from_cloud(c, precision=precision)
    b.substeps(3)
    snap = b.get_state()
    b.destroy()
    r = L.from_cloud(c, precision=precision)
    r.set_state(*snap)
    r.substeps(4)
    got = r.get_state() + r.force()
    r.destroy()
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_expired_wait_is_reported_and_the_context_stays_usable():
    import paper_2606_02711_gb300.lym1 as L
    c = wl.lognormal_cloud(16, 8, seed=42)   # one block of 128 cells
    ctx = L.from_cloud(c, precision=L.MIXED_FAST)
    ctx.substeps(2)
    good = ctx.get_state()
    ctx.debug_expire_wait()
    ctx.substeps(1)
    assert ctx.synchronize_status() == L.ETIMEOUT
    assert ctx.synchronize_status() == L.OK      # reported once
    ctx.set_state(*good)
    ctx.substeps(3)
    assert ctx.synchronize_status() == L.OK
    J, Hx, Hy = ctx.get_state()
    assert np.all(np.isfinite(J)) and J.max() > 0
    ctx.destroy()

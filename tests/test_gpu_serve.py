"""Serving on the GPU: continuous batching gives each cloud the result it gets
alone (FP64_DET, bit for bit), and the loop reports latencies."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def test_result_same_alone_and_in_the_mix():
    import paper_2606_02711_gb300.lym1 as L
    from paper_2606_02711_gb300.serve import Lym1Backend, Request, Server
    edges = oracle.freq_grid()
    A = wl.lognormal_cloud(40, 32, seed=31, mean_nh=2e2, L_sun=1e5, Z=1e-2)
    B = wl.lognormal_cloud(64, 48, seed=32, mean_nh=1e3, L_sun=1e6, Z=1e-3)
    C = wl.lognormal_cloud(24, 24, seed=33, mean_nh=5e2, L_sun=1e4, Z=0.0)
    kw = dict(check_every=20, tol=1e-3, max_substeps=200, keep_force=True)
    alone = Server(Lym1Backend(L.FP64_DET, edges=edges), **kw).run([Request(0, 0.0, A)])
    mix = Server(Lym1Backend(L.FP64_DET, edges=edges), **kw).run(
        [Request(1, 0.0, B), Request(0, 0.02, A), Request(2, 0.03, C)])
    a = alone[0]
    m = {r.rid: r for r in mix}[0]
    assert a.substeps == m.substeps and a.converged == m.converged
    assert np.array_equal(a.force[0], m.force[0]) and np.array_equal(a.force[1], m.force[1])
    for k in ("e_tot", "emitted", "absorbed", "outflow", "work"):
        assert a.diag[k] == m.diag[k], k
    assert len(mix) == 3 and all(r.latency > 0 for r in mix)


@pytest.mark.parametrize("kind", ["plain", "mixed", "gray", "cyl", "temp", "fine"])
def test_plan_bytes_equals_device_bytes(kind):
    import paper_2606_02711_gb300.lym1 as L
    edges = None
    c = wl.lognormal_cloud(45, 38, seed=3)
    prec, q = L.FP64, 0.0
    if kind == "mixed":
        prec = L.MIXED
    elif kind == "gray":
        c = wl.uniform_gray(40, 28)
    elif kind == "cyl":
        c = wl.uniform_sphere(32, tau_cl=1e3)
    elif kind == "temp":
        c.temp = wl.two_phase_temperature(c.nx, c.ny, seed=7, T_cold=80.0, T_hot=2.0e4)
    elif kind == "fine":
        q = 1.03
    ctx = L.from_cloud(c, precision=prec, edges=edges, q=q)
    want = ctx.info()["device_bytes"]
    got = L.plan_bytes(c.nx, c.ny, prec, geometry=c.geometry, q=q, gray=c.gray,
                       temp_field=c.temp is not None)
    ctx.destroy()
    assert got == want


def test_serving_rounds_with_unchanged_membership_reuse_the_batch():
    import paper_2606_02711_gb300.lym1 as L
    from paper_2606_02711_gb300.serve import Lym1Backend, Request, Server
    A = wl.lognormal_cloud(48, 48, seed=41, mean_nh=2e2, L_sun=1e5)
    B = wl.lognormal_cloud(32, 32, seed=42, mean_nh=2e2, L_sun=1e5)
    be = Lym1Backend(L.MIXED)
    srv = Server(be, check_every=10, tol=1e-30, max_substeps=60)
    res = srv.run([Request(0, 0.0, A), Request(1, 0.0, B)])
    # both admitted at once, six rounds of ten substeps, one batch for all of them
    assert len(res) == 2 and srv.rounds == 6
    assert be.batch_creations == 1
    # a new batch of the same class starts with the cached tuned grid
    ca = L.from_cloud(A, precision=L.MIXED)
    cb = L.from_cloud(B, precision=L.MIXED)
    b1 = L.Batch([ca, cb])
    assert b1.grid()[0] > 0
    b1.destroy()
    ca.destroy()
    cb.destroy()

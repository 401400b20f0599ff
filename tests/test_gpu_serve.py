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

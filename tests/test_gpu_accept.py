"""GPU parity of the substep acceptance rule of step 2 (Sec. 2.1 step 2 and its
footnote) against the oracle's rule, through the C ABI.

Bars as in the other parity tests, per element: FP64_DET bit-exact (the
subcycling kernel takes every decision and update in the oracle's operation
order), FP64 1e-10, the FP32-state policies 1e-4 plus the n u S_n floor.  Every case checks that
the oracle subcycled some cells (and not all), so the rule is exercised.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import check_outputs, fw_of

pytestmark = pytest.mark.gpu

TOL = {0: 0.0, 1: 1e-10, 2: 1e-4, 3: 1e-4}


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


def run_pair(L, cloud, precision, nsteps, state=None, dt=None):
    edges = oracle.freq_grid()
    ctx = L.from_cloud(cloud, precision=precision, edges=edges)
    ctx.set_accept(True)
    O = oracle.Oracle(edges=edges, accept=True, **cloud.kwargs())
    O.subcycle_on(True)
    if state is not None:
        ctx.set_state(*state)
    st = state if state is not None else O.zero_state()
    nmax, diags = [], []
    for _ in range(nsteps):
        r = O.substep(*st, dt=dt)
        st = r[:3]
        nmax.append(O.nsub.copy())
        diags.append(r[5])
    if dt is None:
        ctx.substeps(nsteps)
    else:
        for _ in range(nsteps):
            ctx.substeps(1, dt)
    got = ctx.get_state() + ctx.force()
    dg = ctx.diagnostics()
    ctx.destroy()
    # the diagnostics' flows add up over the substeps; the energy is the last
    d = {k: sum(x[k] for x in diags) for k in ("emitted", "absorbed", "outflow", "work")}
    d["e_after"] = diags[-1]["e_after"]
    return got, r[:5], dg, d, np.array(nmax)


def _strong_source_state(c, nb):
    # a populated field, with a source 1e3 times brighter than the field's own
    # level: the source cells change by far more than 10 % in one RT step
    J, Hx, Hy = wl.populated_state(c, nb, J0=1e-13)
    return J, Hx, Hy


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_lognormal_cloud_with_the_rule(L, precision):
    c = wl.lognormal_cloud(45, 38, seed=3, v_edge_kms=30.0, L_sun=1e7)
    st = _strong_source_state(c, 194)
    got, ref, dg, d, nsub = run_pair(L, c, precision, 3, st)
    assert nsub.max() > 1 and np.any(nsub == 1)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c))
    rel = max(TOL[precision], 1e-12)
    assert dg["emitted"] == pytest.approx(d["emitted"], rel=max(rel, 1e-12))
    assert dg["absorbed"] == pytest.approx(d["absorbed"], rel=max(rel, 1e-12))
    assert dg["e_tot"] == pytest.approx(d["e_after"], rel=max(rel, 1e-12))


@pytest.mark.parametrize("precision", [0, 2])
def test_one_substep_path_with_another_dt(L, precision):
    # lym1_substeps with an explicit dt takes the one-launch-per-kernel path
    c = wl.lognormal_cloud(40, 24, seed=4, L_sun=1e7)
    st = _strong_source_state(c, 194)
    O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    dt = 0.7 * O.dt_cfl
    got, ref, dg, d, nsub = run_pair(L, c, precision, 2, st, dt=dt)
    assert nsub.max() > 1
    check_outputs(got, ref, TOL[precision], 2, st, fw_of(c) / 0.7)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_axisymmetric_sphere_from_empty(L, precision):
    c = wl.uniform_sphere(32, tau_cl=1e4)
    got, ref, dg, d, nsub = run_pair(L, c, precision, 3)
    assert nsub.max() > 1
    check_outputs(got, ref, TOL[precision], 3, fw=fw_of(c))
    assert dg["emitted"] == pytest.approx(d["emitted"], rel=max(TOL[precision], 1e-12))


@pytest.mark.parametrize("precision", [0, 2, 3])
def test_gray_group_with_the_rule(L, precision):
    c = wl.uniform_gray(40, 28)
    got, ref, dg, d, nsub = run_pair(L, c, precision, 4)
    assert nsub.max() > 1
    check_outputs(got, ref, TOL[precision], 4, fw=fw_of(c))
    assert dg["e_tot"] == pytest.approx(d["e_after"], rel=max(TOL[precision], 1e-12))


def test_batch_equals_solo_runs(L):
    A = wl.lognormal_cloud(40, 32, seed=31, L_sun=1e6)
    B = wl.lognormal_cloud(24, 24, seed=32, L_sun=1e5)
    solo = []
    for c in (A, B):
        ctx = L.from_cloud(c, precision=L.FP64_DET)
        ctx.set_accept(True)
        ctx.substeps(3)
        solo.append(ctx.get_state() + ctx.force())
        ctx.destroy()
    ca, cb = (L.from_cloud(c, precision=L.FP64_DET) for c in (A, B))
    for ctx in (ca, cb):
        ctx.set_accept(True)
    b = L.Batch([ca, cb])
    b.substeps(3)
    b.destroy()
    for ctx, ref in zip((ca, cb), solo):
        got = ctx.get_state() + ctx.force()
        for a, r in zip(got, ref):
            assert np.array_equal(a, r)
        ctx.destroy()


def test_refusals(L):
    c = wl.lognormal_cloud(16, 16, seed=5)
    aF, ka, je = wl.stellar_bands(c)
    bands = L.Context.for_bands(nx=c.nx, ny=c.ny, dx=c.dx, alpha_F=aF, kappa=ka, emissivity=je)
    with pytest.raises(L.Lym1Error):
        bands.set_accept(True)
    bands.destroy()
    a = L.from_cloud(c, precision=L.MIXED)
    b = L.from_cloud(c, precision=L.MIXED)
    a.set_accept(True)
    with pytest.raises(L.Lym1Error):  # the contexts of a batch share the setting
        L.Batch([a, b])
    b.set_accept(True)
    batch = L.Batch([a, b])
    a.set_accept(False)
    with pytest.raises(L.Lym1Error):  # a batch made before the change refuses to run
        batch.substeps(1)
    batch.destroy()
    a.destroy()
    b.destroy()

"""Active-bin pruning on the GPU (lym1_set_pruning, Sec. 2.2: bins holding no
more than the cut, 1e-10 in the paper, of the domain energy skip step 1)
against the oracle's pruning mode, with the per-element bars of
test_gpu_parity (bit-exact LYM1_FP64_DET, 1e-10 LYM1_FP64, 1e-4 plus the
n u S_n floor for the mixed policies), in both geometries, through the graph-replayed and
batched paths.  The states hold chosen bins at shares of ~1e-14, far from the
cut, so that the two sides never face a borderline decision."""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, close, fw_of

pytestmark = pytest.mark.gpu

CUT = 1e-10


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


def state(nb, ny, nx, seed, small=range(0, 194, 3), f=1e-14):
    g = np.random.default_rng(seed)
    J = 1e-3 * np.exp(g.normal(0, 0.5, (nb, ny, nx)))
    Hx = 0.5 * J * g.uniform(-1, 1, J.shape)
    Hy = 0.5 * J * g.uniform(-1, 1, J.shape)
    for k in small:
        for a in (J, Hx, Hy):
            a[k] *= f
    return J, Hx, Hy


def run_pair(L, c, edges, precision, n, st, prune=CUT):
    ctx = L.from_cloud(c, precision=precision, edges=edges)
    ctx.set_pruning(prune)
    ctx.set_state(*st)
    ctx.substeps(n)
    got = ctx.get_state() + ctx.force()
    dg = ctx.diagnostics()
    ctx.destroy()
    ref, diags = oracle.Oracle(edges=edges, prune=prune, **c.kwargs()).run(n, st)
    return got, ref, dg, diags


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_pruned_substeps_match_oracle(L, edges, precision):
    c = wl.lognormal_cloud(45, 38, seed=171, v_edge_kms=100.0, Z=0.2, p_d=1e-7)
    c.lum = 1e-6 * c.lum  # weak sources: the small bins stay below the cut
    st = state(194, 38, 45, 172)
    got, ref, dg, diags = run_pair(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))
    rel = max(TOL[precision], 1e-12)
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=rel)
    out = sum(x["outflow"] for x in diags)
    assert dg["outflow"] == pytest.approx(out, rel=max(rel, 1e-10))


@pytest.mark.parametrize("precision", [0, 3])
def test_pruning_axisymmetric_vacuum(L, edges, precision):
    c = wl.lognormal_cloud(37, 29, seed=173, v_edge_kms=100.0)
    c.geometry, c.bc = 1, (0, 1, 0, 1)
    c.lum = 1e-6 * c.lum
    st = state(194, 29, 37, 174)
    got, ref, _, _ = run_pair(L, c, edges, precision, 2, st)
    check_outputs(got, ref, TOL[precision], 2, st, fw_of(c, edges))


def test_pruned_bins_stay_put_in_vacuum(L, edges):
    # no gas, no sources, no frequency step: pruned bins come out unchanged
    nx, ny = 40, 24
    z = np.zeros((ny, nx))
    ctx = L.Context(nx=nx, ny=ny, dx=1e16, n_hi=z, rho_d=z, p_d=z, ux=z, uy=z, freq_step=False,
                    edges=edges, precision="mixed_fast", bc=(1, 1, 1, 1))
    ctx.set_pruning(CUT)
    st = state(194, ny, nx, 175)
    ctx.set_state(*st)
    ctx.substeps(1)
    J, Hx, Hy = ctx.get_state()
    ctx.destroy()
    small = list(range(0, 194, 3))
    J32 = st[0].astype(np.float32).astype(np.float64)
    for k in small:
        np.testing.assert_array_equal(J[k], J32[k])
    assert all(not np.array_equal(J[k], J32[k]) for k in range(1, 194, 3))


def test_switching_pruning_on_graph_and_batch_paths(L, edges):
    c = wl.lognormal_cloud(40, 24, seed=176, v_edge_kms=80.0)
    c.lum = 1e-6 * c.lum
    st = state(194, 24, 40, 177)
    ctx = L.from_cloud(c, precision=0, edges=edges)
    ctx.set_state(*st)
    ctx.substeps(2)          # graph path, every bin advected
    ctx.set_pruning(CUT)
    ctx.substeps(2)          # graph path rebuilt with the pruning launches
    got = ctx.get_state()
    O0 = oracle.Oracle(edges=edges, **c.kwargs())
    (J, Hx, Hy, _, _), _ = O0.run(2, st)
    O1 = oracle.Oracle(edges=edges, prune=CUT, **c.kwargs())
    (J, Hx, Hy, _, _), _ = O1.run(2, (J, Hx, Hy))
    for a, b, n in zip(got, (J, Hx, Hy), ("J", "Hx", "Hy")):
        close(a, b, 0.0, n)
    # a batch made before a change of the cut refuses to run; a new one runs
    b = L.Batch([ctx])
    ctx.set_pruning(1e-8)
    with pytest.raises(L.Lym1Error) as e:
        b.substeps(1)
    assert e.value.status == L.EINVAL
    b.destroy()
    b = L.Batch([ctx])
    b.substeps(1)
    b.destroy()
    with pytest.raises(L.Lym1Error) as e:
        ctx.set_pruning(1.0)
    assert e.value.status == L.EINVAL
    ctx.destroy()

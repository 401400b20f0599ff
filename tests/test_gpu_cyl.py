"""GPU parity on the axisymmetric (R, Z) grid (geometry 1): the CUDA path through
the C ABI against the FP64 oracle's cylindrical substep, with the bars of
test_gpu_parity (bit-exact for LYM1_FP64_DET, 1e-10 for LYM1_FP64, 1e-4 per
element plus the n u S_n floor for the mixed policies), plus the thin-sphere force
multiplier tau eta / 4 of Sec. 4.1 (Test 1, optically thin limit)."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, close, fw_of, random_state

pytestmark = pytest.mark.gpu

C = 2.99792458e10


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


def cyl_cloud(nx, ny, seed, v_kms=30.0, **kw):
    """Lognormal cloud on the (R, Z) grid with u = v (R, Z) / r_max from the
    origin and the source in the cells next to the axis at the midplane."""
    c = wl.lognormal_cloud(nx, ny, seed=seed, **kw)
    c.geometry = 1
    R = (np.arange(nx) + 0.5) * c.dx
    Z = (np.arange(ny) + 0.5) * c.dx
    RR, ZZ = np.meshgrid(R, Z)
    rmax = math.hypot(R[-1], Z[-1])
    c.ux = v_kms * wl.KM * RR / rmax
    c.uy = v_kms * wl.KM * ZZ / rmax
    lum = np.zeros((ny, nx))
    lum[0, 0] = lum[0, min(1, nx - 1)] = lum[min(1, ny - 1), 0] = 1e39
    c.lum = lum
    return c


def run_both(L, cloud, edges, precision, nsteps, state=None):
    ctx = L.from_cloud(cloud, precision=precision, edges=edges)
    O = oracle.Oracle(edges=edges, **cloud.kwargs())
    if state is not None:
        ctx.set_state(*state)
    ctx.substeps(nsteps)
    got = ctx.get_state() + ctx.force()
    dg = ctx.diagnostics()
    ref, diags = O.run(nsteps, state)
    ctx.destroy()
    return got, ref, dg, diags


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_cyl_gray_sphere(L, edges, precision):
    # gray uniform sphere (tau_cl = 30), ragged 40 x 28 cut, from zero
    s = wl.uniform_sphere(40, tau_cl=30.0, gray=True)
    s.ny = 28
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        setattr(s, f, np.ascontiguousarray(getattr(s, f)[:28, :]))
    got, ref, dg, diags = run_both(L, s, edges, precision, 25)
    check_outputs(got, ref, TOL[precision], 25, fw=fw_of(s, edges))
    d = diags[-1]
    rel = max(TOL[precision], 1e-12)
    assert dg["e_tot"] == pytest.approx(d["e_after"], rel=rel)
    assert dg["force_abs"] == pytest.approx(d["force_abs"], rel=max(rel, 1e-12))
    assert dg["force_radial"] == pytest.approx(d["force_radial"], rel=max(rel, 1e-12))


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_cyl_lognormal_194_bins(L, edges, precision):
    # dust, destruction, Hubble-like flow from the origin (hoop work term),
    # recoil, random state with H_R != 0 at the axis; several tiles + tails
    c = cyl_cloud(45, 38, seed=13)
    st = random_state(194, 38, 45, 17)
    got, ref, dg, diags = run_both(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))
    rel = max(TOL[precision], 1e-12)
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=rel)
    keys = ("emitted", "absorbed", "work", "outflow")
    ref_sums = {k: sum(x[k] for x in diags) for k in keys}
    scale = max(abs(v) for v in ref_sums.values())
    for k in keys:
        assert abs(dg[k] - ref_sums[k]) <= max(rel, 1e-10) * scale, k


def test_cyl_velocity_extremes_and_vacuum(L, edges):
    c = cyl_cloud(33, 17, seed=14, v_kms=2000.0)
    c.n_hi[5:9, 10:20] = 0.0
    c.ux[:, :10] *= -1.0
    got, ref, _, _ = run_both(L, c, edges, 0, 2, random_state(194, 17, 33, 18))
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 0.0, n)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (2, 3), (32, 8), (33, 9)])
def test_cyl_degenerate_and_ragged_shapes(L, edges, shape):
    nx, ny = shape
    c = cyl_cloud(max(nx, 2), max(ny, 2), seed=15)
    c.nx, c.ny = nx, ny
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        setattr(c, f, np.ascontiguousarray(getattr(c, f)[:ny, :nx]))
    c.lum[...] = 1e36
    got, ref, _, _ = run_both(L, c, edges, 0, 2, random_state(194, ny, nx, 19))
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 0.0, n)


def test_cyl_batch_matches_solo_and_rejects_mixed_geometry(L, edges):
    clouds = [cyl_cloud(40, 24, seed=20), cyl_cloud(17, 33, seed=21)]
    solo = []
    for c in clouds:
        x = L.from_cloud(c, precision="mixed_fast", edges=edges)
        for _ in range(6):
            x.substeps(1)
        solo.append(x.get_state())
        x.destroy()
    ctxs = [L.from_cloud(c, precision="mixed_fast", edges=edges) for c in clouds]
    b = L.Batch(ctxs)
    b.substeps(6)
    b.destroy()
    for x, s in zip(ctxs, solo):
        for a, r in zip(x.get_state(), s):
            np.testing.assert_array_equal(a, r)
        x.destroy()
    cart = wl.lognormal_cloud(16, 16, seed=22)
    a = L.from_cloud(cart, precision="mixed_fast", edges=edges)
    bcyl = L.from_cloud(clouds[0], precision="mixed_fast", edges=edges)
    with pytest.raises(L.Lym1Error) as e:
        L.Batch([a, bcyl])
    assert e.value.status == L.EINVAL
    a.destroy()
    bcyl.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fast"])
def test_cyl_thin_sphere_force_multiplier(L, edges, precision):
    # Sec. 4.1, Test 1: M_F -> tau_cl eta / 4 for an optically thin uniform
    # sphere with uniform emission (steady state, 12 light-crossing times)
    s = wl.uniform_sphere(32, tau_cl=0.1, gray=True)
    ctx = L.from_cloud(s, precision=precision, edges=edges)
    R_cl = s.meta["R_cl"]
    ctx.substeps(int(60 * R_cl / s.dx))
    d = ctx.diagnostics()
    ctx.destroy()
    lc = oracle.line_constants(s.T)
    eta = oracle.bin_tables(edges, s.T)["eta"]
    tau = float(s.n_hi.max()) * lc["sigma0"] * R_cl
    mf = d["force_abs"] / (s.L_total / C)
    assert abs(mf / (tau * eta / 4.0) - 1.0) < 0.02
    assert abs(d["force_radial"] / d["force_abs"] - 1.0) < 2e-3


@pytest.mark.parametrize("precision", [0, 3])
def test_cyl_vacuum_outer_edges(L, edges, precision):
    c = cyl_cloud(37, 29, seed=33)
    c.bc = (0, 1, 0, 1)
    st = random_state(194, 29, 37, 34)
    got, ref, _, _ = run_both(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))

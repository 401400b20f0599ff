"""Broad bands on the GPU (Sec. 3: the seven stellar and IR bands on the M1
transport of Sec. 2.1 without frequency terms) through lym1_create_bands,
against the oracle's band mode with the bars of test_gpu_parity (bit-exact
LYM1_FP64_DET, 1e-10 LYM1_FP64, 1e-4 per element plus the n u S_n floor for
the mixed policies), in both geometries with vacuum sides, with emergent spectra, across
an update of the opacities, and reduced to the gray Lya group bit for bit.
The thin-sphere force multiplier tau / 4 (Sec. 4.1, Test 1, thin limit, eta = 1
for a band) is checked on the GPU too."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, close, force_weights, random_state

pytestmark = pytest.mark.gpu

C = 2.99792458e10


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


def band_cloud(nx, ny, seed, geometry=0, v_kms=200.0):
    c = wl.lognormal_cloud(nx, ny, seed=seed, v_edge_kms=v_kms, Z=0.3, box_pc=0.5)
    c.geometry = geometry
    c.bc = (0, 1, 0, 1) if geometry == 1 else (1, 1, 1, 1)
    return c, wl.stellar_bands(c)


def run_pair(L, c, bands, precision, n, state):
    aF, ka, je = bands
    kw = dict(nx=c.nx, ny=c.ny, dx=c.dx, ux=c.ux, uy=c.uy, geometry=c.geometry, bc=c.bc)
    ctx = L.Context.for_bands(alpha_F=aF, kappa=ka, emissivity=je, precision=precision, **kw)
    O = oracle.Oracle.for_bands(alpha_F=aF, kappa=ka, emissivity=je, **kw)
    assert ctx.nb == 7 and ctx.dt_cfl == O.dt_cfl
    ctx.set_state(*state)
    ctx.substeps(n)
    got = ctx.get_state() + ctx.force()
    dg = ctx.diagnostics()
    ref, diags = O.run(n, state)
    return ctx, O, got, ref, dg, diags


@pytest.mark.parametrize("geometry", [0, 1])
@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_seven_bands_match_oracle(L, precision, geometry):
    c, bands = band_cloud(45, 38, seed=101, geometry=geometry)
    st = random_state(7, 38, 45, 102, scale=1e-3)
    ctx, O, got, ref, dg, diags = run_pair(L, c, bands, precision, 4, st)
    ctx.destroy()
    check_outputs(got, ref, TOL[precision], 4, st, force_weights(O, c.dx))
    rel = max(TOL[precision], 1e-12)
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=rel)
    keys = ("emitted", "absorbed", "work", "outflow")
    ref_sums = {k: sum(x[k] for x in diags) for k in keys}
    scale = max(abs(v) for v in ref_sums.values())
    for k in keys:
        assert abs(dg[k] - ref_sums[k]) <= max(rel, 1e-10) * scale, k


@pytest.mark.parametrize("precision", [0, 3])
def test_band_update_and_spectrum(L, precision):
    c, bands = band_cloud(37, 29, seed=103)
    aF, ka, je = bands
    st = random_state(7, 29, 37, 104, scale=1e-3)
    kw = dict(nx=c.nx, ny=c.ny, dx=c.dx, ux=c.ux, uy=c.uy, geometry=0, bc=c.bc)
    ctx = L.Context.for_bands(alpha_F=aF, kappa=ka, emissivity=je, precision=precision, **kw)
    ctx.set_state(*st)
    ctx.spectrum_enable()
    ctx.substeps(2)
    # the opacities of an ionised core (EUV absorption gone), then two more substeps
    aF2, ka2 = aF.copy(), ka.copy()
    core = (slice(None), slice(10, 19), slice(14, 23))
    aF2[core] = 0.1 * aF2[core]
    ka2[core] = 0.1 * ka2[core]
    ctx.bands_update(aF2, ka2, 2.0 * je)
    ctx.substeps(2)
    got = ctx.get_state() + ctx.force()
    spec = ctx.spectrum()
    ctx.destroy()
    O1 = oracle.Oracle.for_bands(alpha_F=aF, kappa=ka, emissivity=je, **kw)
    O2 = oracle.Oracle.for_bands(alpha_F=aF2, kappa=ka2, emissivity=2.0 * je, **kw)
    J, Hx, Hy = st
    ref_spec = 0.0
    for O in (O1, O1, O2, O2):
        O.spectrum_on()
        J, Hx, Hy, fx, fy, _ = O.substep(J, Hx, Hy)
        ref_spec = ref_spec + O.spectrum
    check_outputs(got, (J, Hx, Hy, fx, fy), TOL[precision], 4, st, force_weights(O1, c.dx))
    if precision == 0:
        np.testing.assert_array_equal(spec, ref_spec)
    else:
        scale = np.abs(ref_spec).max(axis=1, keepdims=True)
        assert np.all(np.abs(spec - ref_spec) <= 1e-4 * scale + 1e-300)


def test_band_with_gray_group_inputs_is_the_gray_group(L):
    c = wl.lognormal_cloud(40, 28, seed=105, Z=0.5, p_d=1e-6, v_edge_kms=300.0)
    c.gray = True
    gray = L.from_cloud(c, precision=0, edges=oracle.freq_grid())
    alpha = c.n_hi * gray.info()["sigma0"]
    aH = alpha * gray.info()["eta"]
    aF = (aH + c.rho_d * c.kappa_F)[None]
    ka = (c.rho_d * c.kappa_abs + c.p_d * aH)[None]
    je = (c.lum * (1.0 / ((4.0 * math.pi) * ((c.dx * c.dx) * c.dx))))[None]
    band = L.Context.for_bands(nx=c.nx, ny=c.ny, dx=c.dx, ux=c.ux, uy=c.uy, alpha_F=aF, kappa=ka,
                               emissivity=je, precision=0)
    st = random_state(1, 28, 40, 106, scale=1e-3)
    for x in (gray, band):
        x.set_state(*st)
        x.substeps(5)
    for u, w, n in zip(gray.get_state() + gray.force(), band.get_state() + band.force(),
                       ("J", "Hx", "Hy", "fx", "fy")):
        close(u, w, 0.0, n)
    gray.destroy()
    band.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fast"])
def test_thin_sphere_band_force_multiplier(L, precision):
    n, tau = 32, 0.1
    s = wl.uniform_sphere(n, tau_cl=tau, gray=True)
    R = s.meta["R_cl"]
    inside = s.n_hi > 0
    aF = np.where(inside, tau / R, 0.0)[None]
    j = np.where(inside, 1e-22, 0.0)[None]
    ctx = L.Context.for_bands(nx=n, ny=n, dx=s.dx, alpha_F=aF, kappa=np.zeros_like(aF),
                              emissivity=j, geometry=1, bc=(0, 1, 0, 1), precision=precision)
    ctx.substeps(int(60 * R / s.dx))
    d = ctx.diagnostics()
    ctx.destroy()
    ring = math.pi * (2.0 * np.arange(n) + 1.0) * s.dx ** 3
    Lh = (4.0 * math.pi * j[0] * ring[None, :]).sum()
    assert d["L_tot"] == pytest.approx(Lh, rel=1e-12)
    assert abs(d["M_F"] / (tau / 4.0) - 1.0) < 0.02
    assert abs(d["force_radial"] / d["force_abs"] - 1.0) < 2e-3


def test_band_context_rejects(L):
    c, (aF, ka, je) = band_cloud(16, 16, seed=107)
    kw = dict(nx=16, ny=16, dx=c.dx, ux=c.ux, uy=c.uy)
    for bad in ("neg", "nan"):
        a = aF.copy()
        a[3, 4, 5] = -1.0 if bad == "neg" else float("nan")
        with pytest.raises(L.Lym1Error) as e:
            L.Context.for_bands(alpha_F=a, kappa=ka, emissivity=je, precision=3, **kw)
        assert e.value.status == L.EINVAL
    ctx = L.Context.for_bands(alpha_F=aF, kappa=ka, emissivity=je, precision=3, **kw)
    ctx.substeps(2)
    before = ctx.get_state()
    k2 = ka.copy()
    k2[0, 0, 0] = float("inf")
    for call in (lambda: ctx.bands_update(aF, k2, je), lambda: ctx.set_sources(c.lum),
                 lambda: ctx.dynamic_ctilde(), lambda: L.Batch([ctx])):
        with pytest.raises(L.Lym1Error) as e:
            call()
        assert e.value.status == L.EINVAL
    for u, w in zip(ctx.get_state(), before):
        np.testing.assert_array_equal(u, w)
    ctx.destroy()

"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (one context, the default stream, CFL substeps), with the
per-element bars of test_gpu_parity:

* uniform-gray 64x64: all 2000 substeps, FP64_DET, bit-exact;
* lognormal-512 (512x512x194) from a populated realisable state (every cell
  and bin holds radiation, |H| < J): FP64_DET bit-exact after 2 substeps,
  MIXED and MIXED_FAST after 5, against the oracle on the full grid;
* the seven stellar/IR bands on lognormal-512 from a populated state:
  FP64_DET bit-exact and MIXED_FAST after 10 substeps, on the full grid;
* a 128x128x194 crop of lognormal-512, MIXED and MIXED_FAST, 200 substeps
  from a populated state and from the empty state (errors accumulated over
  hundreds of substeps, as in steady-state and served runs);
* lognormal-2048 (2048x2048x194), MIXED_FAST: 5 substeps from the empty
  state; the oracle computes the central 64x64 crop, which the radiation
  cannot leave in 5 substeps (the stencil reaches 2 cells per substep), so
  every crop cell is comparable.
"""
import copy

import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, force_weights, fw_of, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


def crop(full, n):
    """The central n x n cells of a cloud, as a cloud of its own."""
    j0 = (full.ny - n) // 2
    c = copy.copy(full)
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        setattr(c, f, np.ascontiguousarray(getattr(full, f)[j0:j0 + n, j0:j0 + n]))
    c.nx = c.ny = n
    return c


def test_uniform_gray_64_all_2000_substeps_bitexact(L):
    c = wl.uniform_gray()
    ctx = L.from_cloud(c, precision=L.FP64_DET, edges=oracle.freq_grid())
    ctx.substeps(2000)
    got = ctx.get_state() + ctx.force()
    O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    ref, diags = O.run(2000)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        assert np.array_equal(a, b), n
    d = ctx.diagnostics()
    assert d["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=1e-12)
    ctx.destroy()


@pytest.fixture(scope="module")
def lognormal_512():
    c = wl.config_lognormal_512()
    return c, wl.populated_state(c, 194, seed=11)


def test_lognormal_512_fp64_det_bitexact(L, lognormal_512):
    c, st = lognormal_512
    ctx = L.from_cloud(c, precision=L.FP64_DET)
    ctx.set_state(*st)
    ctx.substeps(2)
    got = ctx.get_state() + ctx.force()
    ctx.destroy()
    O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    ref, _ = O.run(2, st)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        assert np.array_equal(a, b), n


@pytest.mark.parametrize("precision", [2, 3])
def test_lognormal_512_mixed_policies(L, lognormal_512, precision):
    c, st = lognormal_512
    ctx = L.from_cloud(c, precision=precision)
    ctx.set_state(*st)
    ctx.substeps(5)
    got = ctx.get_state() + ctx.force()
    d = ctx.diagnostics()
    ctx.destroy()
    O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    ref, diags = O.run(5, st)
    check_outputs(got, ref, TOL[precision], 5, st, force_weights(O, c.dx))
    assert d["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=1e-5)
    assert d["max_f"] < 2.0


@pytest.fixture(scope="module")
def crop_runs():
    """Oracle results on the 128^2 crop after 1 and 200 substeps, from the
    populated state and from the empty state."""
    c = crop(wl.config_lognormal_512(), 128)
    O = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    out = {}
    for start in ("populated", "empty"):
        st = wl.populated_state(c, 194, seed=12) if start == "populated" else None
        r1, d1 = O.run(1, st)
        r200, d200 = O.run(199, r1[:3])
        out[start] = (st, {1: (r1, d1[-1]), 200: (r200, d200[-1])})
    return c, out


@pytest.mark.parametrize("start", ["populated", "empty"])
@pytest.mark.parametrize("precision", [2, 3])
def test_crop_128_200_substeps(L, crop_runs, precision, start):
    c, out = crop_runs
    st, refs = out[start]
    ctx = L.from_cloud(c, precision=precision)
    if st is not None:
        ctx.set_state(*st)
    done = 0
    for n in (1, 200):
        ctx.substeps(n - done)
        done = n
        ref, dref = refs[n]
        check_outputs(ctx.get_state() + ctx.force(), ref, TOL[precision], n, st, fw_of(c))
        d = ctx.diagnostics()
        assert d["e_tot"] == pytest.approx(dref["e_after"], rel=1e-4)
        if dref["force_abs"] > 0.0:
            assert d["force_abs"] == pytest.approx(dref["force_abs"], rel=1e-4)
    ctx.destroy()


@pytest.mark.parametrize("precision", ["fp64_det", "mixed_fast"])
def test_seven_bands_lognormal_512(L, precision):
    # the bench's band line: the seven stellar/IR bands on lognormal-512,
    # against the oracle's band mode on the full grid (FP64_DET bit-exact)
    c = wl.config_lognormal_512()
    aF, ka, je = wl.stellar_bands(c)
    kw = dict(nx=c.nx, ny=c.ny, dx=c.dx, ux=c.ux, uy=c.uy)
    st = random_state(7, c.ny, c.nx, 21, scale=1e-3)
    ctx = L.Context.for_bands(alpha_F=aF, kappa=ka, emissivity=je, precision=precision, **kw)
    ctx.set_state(*st)
    ctx.substeps(10)
    got = ctx.get_state() + ctx.force()
    ctx.destroy()
    O = oracle.Oracle.for_bands(alpha_F=aF, kappa=ka, emissivity=je, **kw)
    ref, _ = O.run(10, st)
    if precision == "fp64_det":
        for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
            assert np.array_equal(a, b), n
    else:
        check_outputs(got, ref, TOL[3], 10, st, force_weights(O, c.dx))


def test_lognormal_2048_mixed_fast_central_crop(L):
    c = wl.config_lognormal_2048()
    ctx = L.from_cloud(c, precision=L.MIXED_FAST)
    dt = ctx.dt_cfl
    ctx.substeps(5)
    J, Hx, Hy = ctx.get_state()
    fx, fy = ctx.force()
    ctx.destroy()
    n = 64
    j0 = (c.ny - n) // 2
    sl = (slice(j0, j0 + n), slice(j0, j0 + n))
    kw = c.kwargs()
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        kw[f] = np.ascontiguousarray(kw[f][sl])
    kw["nx"] = kw["ny"] = n
    O = oracle.Oracle(edges=oracle.freq_grid(), **kw)
    ref, _ = O.run(5, dt=dt)
    got = tuple(np.ascontiguousarray(x) for x in
                (J[:, sl[0], sl[1]], Hx[:, sl[0], sl[1]], Hy[:, sl[0], sl[1]], fx[sl], fy[sl]))
    # the radiation has not reached the crop margin: outside it the GPU state is empty
    mask = np.ones(J.shape[1:], bool)
    mask[sl] = False
    assert not J[:, mask].any()
    check_outputs(got, ref, TOL[3], 5, fw=force_weights(O, c.dx))

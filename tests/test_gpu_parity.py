"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars, per element:
  LYM1_FP64_DET   bit-exact (same operation order, no FMA, same exp/expm1)
  LYM1_FP64       |a - b| <= 1e-10 |b| + 1e-12 max|b|
  LYM1_MIXED      |a - b| <= 1e-4 |b| + n u S_n(cell), with u = 2^-24 (the FP32
  LYM1_MIXED_FAST unit roundoff) and n the substeps run.  S_n is the largest
                  magnitude the element's value depends on: the maximum of
                  |J|, |H_x|, |H_y| over every bin of the cells within 2n cells
                  (the domain of dependence of n substeps: the face stencil
                  reaches two cells, the frequency step couples a cell's bins),
                  taken over the reference result and the initial state.  For
                  the force f = 4 pi / (c c_tilde dt) sum_k dnu_k (H' - H''),
                  S_n is the same maximum of Phi = 4 pi / (c c_tilde dt)
                  sum_k dnu_k max(|J_k|, |H_k|): the force of the cell's
                  radiation if all of it were absorbed as flux in one step.
                  The floor states that each substep adds at most one FP32
                  rounding of the largest value a result depends on; it
                  matters only where a value is a small difference of larger
                  terms (a steep front, a flux divergence, a far-wing bin, the
                  small net flux H of a diffusive region that sets the force).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {0: 0.0, 1: 1e-10, 2: 1e-4, 3: 1e-4}


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


U32 = 2.0 ** -24  # FP32 unit roundoff


def dod_max(a2, n):
    """Maximum of a [ny][nx] field over the cells within Chebyshev radius 2n
    of each cell (the reach of n substeps)."""
    from scipy.ndimage import maximum_filter
    r = min(2 * max(int(n), 1), max(a2.shape))
    return maximum_filter(a2, size=2 * r + 1, mode="nearest")


C_LIGHT = 2.99792458e10


def force_weights(src, dx, cfl=0.4, dt_scale=1.0):
    """Per-bin weights 4 pi dnu_k / (c c_tilde dt) of the force sum, with
    c_tilde dt = (CFL / 2) dx (times dt_scale for a substep shorter than the
    CFL one); src is an oracle or a context (anything with tables())."""
    dnu = np.asarray(src.tables()["dnu"], dtype=np.float64)
    return 4.0 * np.pi * dnu / (C_LIGHT * 0.5 * cfl * dx * dt_scale)


def mixed_scales(ref, n, init=None, fw=None):
    """Floor scales of the mixed bar: S_n for the state and, given the force
    weights fw, S_n of Phi for the force."""
    m3 = np.maximum(np.abs(ref[0]), np.maximum(np.abs(ref[1]), np.abs(ref[2])))
    if init is not None:
        for x in init:
            m3 = np.maximum(m3, np.abs(x))
    S = dod_max(m3.max(axis=0), n)
    F = None
    if len(ref) > 3:
        assert fw is not None, "the force bar needs the force weights"
        F = dod_max(np.tensordot(np.asarray(fw), m3, axes=(0, 0)), n)
    return S, F


def close(a, b, rtol, name="", scale=None, n=1):
    if rtol >= 1e-6:
        # elementwise with the floor n u S_n (scale: S_n of a [ny][nx] field)
        assert scale is not None, f"{name}: the mixed bar needs the floor scale"
        floor = n * U32 * (scale[None] if a.ndim == 3 else scale)
        excess = np.abs(a - b) - (rtol * np.abs(b) + floor)
        if np.any(excess > 0):
            i = np.unravel_index(np.argmax(excess), a.shape)
            fl = np.broadcast_to(floor, a.shape)[i]
            raise AssertionError(f"{name}: {int(np.sum(excess > 0))} of {a.size} elements beyond "
                                 f"the bar; worst at {i}: {a[i]!r} vs {b[i]!r} (floor {fl:.3e}, "
                                 f"rtol {rtol})")
        return
    if rtol == 0.0:
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            i = tuple(bad[0])
            raise AssertionError(f"{name}: {bad.shape[0]} of {a.size} differ; first at {i}: "
                                 f"{a[i]!r} vs {b[i]!r}")
        return
    floor = 1e-12 * np.max(np.abs(b)) if b.size else 0.0
    err = np.abs(a - b) - (rtol * np.abs(b) + floor)
    if np.any(err > 0):
        i = np.unravel_index(np.argmax(err), a.shape)
        raise AssertionError(f"{name}: max excess at {i}: {a[i]!r} vs {b[i]!r} (rtol {rtol})")


NAMES = ("J", "Hx", "Hy", "fx", "fy")


def check_outputs(got, ref, rtol, n, init=None, fw=None):
    """(J, Hx, Hy[, fx, fy]) against the reference at one policy's bar after n
    substeps from the state init (None: the empty state); fw: the force
    weights (force_weights) for the mixed bar of the force."""
    S, F = mixed_scales(ref, n, init, fw) if rtol >= 1e-6 else (None, None)
    for i, (a, b) in enumerate(zip(got, ref)):
        close(a, b, rtol, NAMES[i], scale=S if i < 3 else F, n=n)


def random_state(nb, ny, nx, seed, scale=1e-12):
    g = np.random.default_rng(seed)
    J = scale * np.exp(g.normal(0, 1.0, (nb, ny, nx)))
    th = g.uniform(0, 2 * np.pi, (nb, ny, nx))
    f = g.uniform(0, 0.95, (nb, ny, nx))
    return J, J * f * np.cos(th), J * f * np.sin(th)


def fw_of(cloud, edges=None):
    """Force weights of a cloud's problem on a frequency grid (the oracle's
    tables)."""
    O = oracle.Oracle(edges=edges if edges is not None else oracle.freq_grid(), **cloud.kwargs())
    return force_weights(O, cloud.dx, getattr(cloud, "cfl", 0.4))


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


def test_tables_match_oracle(L, edges):
    c = wl.lognormal_cloud(8, 8, seed=1)
    ctx = L.from_cloud(c, precision=L.FP64_DET, edges=edges)
    O = oracle.Oracle(edges=edges, **c.kwargs())
    a, b = ctx.tables(), O.tables()
    for k in ("dnu", "nubar", "Havg", "gem"):
        close(a[k], b[k], 0.0, k)
    assert ctx.dt_cfl == O.dt_cfl
    # default grid (NULL edges) is the paper grid
    ctx2 = L.Context(nx=4, ny=4, dx=c.dx, n_hi=1e3, rho_d=0, p_d=0, ux=0, uy=0)
    assert ctx2.nb == 194
    close(ctx2.tables()["Havg"], b["Havg"], 0.0, "default grid")


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_gray_uniform_cloud(L, edges, precision):
    # the 64x64 uniform gray cloud, ragged 40x28 cut of it, from zero
    c = wl.uniform_gray(40, 28)
    got, ref, dg, diags = run_both(L, c, edges, precision, 25)
    check_outputs(got, ref, TOL[precision], 25, fw=fw_of(c, edges))
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=max(TOL[precision], 1e-12))


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_lognormal_cloud_194_bins(L, edges, precision):
    # lognormal n_H, dust, destruction, v ~ r and recoil; several tiles + tail
    c = wl.lognormal_cloud(45, 38, seed=3, v_edge_kms=30.0)
    st = random_state(194, 38, 45, 7)
    got, ref, dg, diags = run_both(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))
    d = diags[-1]
    assert dg["e_tot"] == pytest.approx(d["e_after"], rel=max(TOL[precision], 1e-12))
    em = sum(x["emitted"] for x in diags)
    ab = sum(x["absorbed"] for x in diags)
    assert dg["emitted"] == pytest.approx(em, rel=max(TOL[precision], 1e-12))
    assert dg["absorbed"] == pytest.approx(ab, rel=max(TOL[precision], 1e-12))


def test_velocity_extremes_and_vacuum_cells(L, edges):
    # large Peclet numbers (fast flow), contracting and expanding regions and
    # cells without H I (no frequency step there)
    c = wl.lognormal_cloud(33, 17, seed=4, v_edge_kms=2000.0)
    c.n_hi[5:9, 10:20] = 0.0
    c.ux[:, :10] *= -1.0
    st = random_state(194, 17, 33, 8)
    got, ref, _, _ = run_both(L, c, edges, 0, 2, st)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 0.0, n)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (2, 3), (32, 8), (33, 9)])
def test_degenerate_and_ragged_shapes(L, edges, shape):
    nx, ny = shape
    c = wl.lognormal_cloud(max(nx, 2), max(ny, 2), seed=5)
    c.nx, c.ny = nx, ny
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        setattr(c, f, np.ascontiguousarray(getattr(c, f)[:ny, :nx]))
    c.lum[...] = 1e36
    got, ref, _, _ = run_both(L, c, edges, 0, 2, random_state(194, ny, nx, 9))
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 0.0, n)


def test_no_sources_stays_zero_and_state_roundtrip(L, edges):
    c = wl.lognormal_cloud(20, 12, seed=6)
    c.lum[...] = 0.0
    ctx = L.from_cloud(c, precision=L.FP64_DET, edges=edges)
    ctx.substeps(4)
    J, Hx, Hy = ctx.get_state()
    assert not J.any() and not Hx.any() and not Hy.any()
    st = random_state(194, 12, 20, 10)
    ctx.set_state(*st)
    back = ctx.get_state()
    for a, b in zip(back, st):
        close(a, b, 0.0)
    E, Fx, Fy = ctx.moments()
    close(E, 4 * np.pi / 2.99792458e10 * st[0], 1e-15)
    close(Fx, 4 * np.pi * st[1], 1e-15)
    ctx.destroy()


def test_step_splits_into_cfl_substeps(L, edges):
    c = wl.lognormal_cloud(16, 16, seed=2)
    ctx = L.from_cloud(c, precision=L.FP64_DET, edges=edges)
    n = ctx.step(3.5 * ctx.dt_cfl)
    assert n == 4
    assert ctx.info()["substeps_done"] == 4
    O = oracle.Oracle(edges=edges, **c.kwargs())
    ref, _ = O.run(4, dt=3.5 * O.dt_cfl / 4)
    close(ctx.get_state()[0], ref[0], 0.0, "J")
    ctx.destroy()


def test_invalid_arguments(L):
    with pytest.raises(L.Lym1Error) as e:
        L.Context(nx=0, ny=4, dx=1.0, n_hi=1.0, rho_d=0, p_d=0, ux=0, uy=0)
    assert e.value.status == L.EINVAL
    with pytest.raises(L.Lym1Error):
        L.Context(nx=4, ny=4, dx=-1.0, n_hi=1.0, rho_d=0, p_d=0, ux=0, uy=0)
    with pytest.raises(L.Lym1Error):
        L.Context(nx=4, ny=4, dx=1.0, n_hi=1.0, rho_d=0, p_d=0, ux=0, uy=0, precision=7)
    with pytest.raises(L.Lym1Error):
        L.Context(nx=4, ny=4, dx=1.0, n_hi=1.0, rho_d=0, p_d=0, ux=0, uy=0,
                  edges=[0.0, 1.0, 1.0])


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_causality_cap_on_unrealisable_input(L, edges, precision):
    # states with |H|/J up to 3 (Sec. 2.1 step 3 leaves |H| <= J in every
    # cell, with or without H I); parity with the oracle at each policy's bar
    c = wl.lognormal_cloud(37, 21, seed=12, v_edge_kms=50.0)
    c.n_hi[3:7, 4:12] = 0.0
    J, Hx, Hy = random_state(194, 21, 37, 23)
    g = np.random.default_rng(24)
    boost = np.where(g.uniform(size=J.shape) < 0.3, g.uniform(1.0, 3.0 / 0.95, J.shape), 1.0)
    st = (J, Hx * boost, Hy * boost)
    got, ref, dg, _ = run_both(L, c, edges, precision, 1, st)
    check_outputs(got, ref, TOL[precision], 1, st, fw_of(c, edges))
    Jg, Hxg, Hyg = got[:3]
    assert np.all(np.hypot(Hxg, Hyg) <= Jg * (1 + (1e-6 if precision >= 2 else 1e-15)))


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 0, 0, 1)])
@pytest.mark.parametrize("precision", [0, 3])
def test_vacuum_outflow_sides(L, edges, bc, precision):
    # outflow into vacuum on some sides (ghosts without radiation), with an
    # inward-pointing random state at the edges
    c = wl.lognormal_cloud(41, 19, seed=31, v_edge_kms=40.0)
    c.bc = bc
    st = random_state(194, 19, 41, 32)
    got, ref, dg, diags = run_both(L, c, edges, precision, 2, st)
    check_outputs(got, ref, TOL[precision], 2, st, fw_of(c, edges))
    out = sum(d["outflow"] for d in diags)
    assert dg["outflow"] == pytest.approx(out, rel=max(TOL[precision], 1e-10))

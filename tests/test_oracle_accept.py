"""Oracle pins for the substep acceptance rule of step 2 (Sec. 2.1 step 2 and
its footnote): a trial emission/absorption substep of a cell is kept when the
cell's Lya energy density changes by |e'' - e'| / (e' + e_floor) < 0.1, with
e_floor = 4 pi J_floor / c and J_floor = 1e-15 erg cm^-2 s^-1 sr^-1; otherwise
it is halved and redone, until the accepted substeps fill the RT step.

Readings (the paper gives the halving only): every cell starts each RT step
with the whole step; after an accepted substep the next trial doubles it,
capped by what is left; substeps are whole multiples of dt / 2^40.

The brute force below is written from that text alone, with plain Python
floats: on a 1x1 grid with zero-gradient edges and no flow, step 1 leaves a
uniform state unchanged (the face fluxes cancel), so a substep with the
frequency step off is step 2 alone.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl

C_LIGHT = 2.99792458e10
J_FLOOR = 1e-15


def brute_step2(J, Hx, Hy, dnu, kap, aF, js, dt, ct):
    """The rule on one cell, bins in order; returns the new state, the accepted
    substep lengths and the force / emission / absorption sums."""
    J, Hx, Hy = list(J), list(Hx), list(Hy)
    nb = len(J)
    full = 2 ** 40
    done, size = 0, full
    e_cur = sum(dnu[k] * J[k] for k in range(nb))
    steps, ax, ay, em, ab = [], 0.0, 0.0, 0.0, 0.0
    while done < full:
        size = min(size, full - done)
        h = dt * (size / full)
        ch = ct * h
        new = [(J[k] + ch * js[k]) / (1.0 + ch * kap[k]) for k in range(nb)]
        e_new = sum(dnu[k] * new[k] for k in range(nb))
        if not (abs(e_new - e_cur) / (e_cur + J_FLOOR) < 0.1) and size > 1:
            size //= 2
            continue
        for k in range(nb):
            hx2 = Hx[k] / (1.0 + ch * aF[k])
            hy2 = Hy[k] / (1.0 + ch * aF[k])
            ax += dnu[k] * (Hx[k] - hx2)
            ay += dnu[k] * (Hy[k] - hy2)
            em += dnu[k] * (ch * js[k])
            ab += dnu[k] * (ch * (kap[k] * new[k]))
            J[k], Hx[k], Hy[k] = new[k], hx2, hy2
        steps.append(h)
        e_cur = e_new
        done += size
        size *= 2
    return np.array(J), np.array(Hx), np.array(Hy), steps, ax, ay, em, ab


def one_cell(n_hi, rho_d, p_d, lum, geometry=0, edges=None, T=1.0e4, kabs=wl.KAPPA_ABS,
             kF=wl.KAPPA_F, dx=1e16):
    edges = oracle.freq_grid() if edges is None else edges
    kw = dict(nx=1, ny=1, dx=dx, edges=edges, T=T, n_hi=n_hi, rho_d=rho_d, p_d=p_d, ux=0.0,
              uy=0.0, lum=lum, kappa_abs=kabs, kappa_F=kF, recoil=False, freq_step=False,
              geometry=geometry)
    return kw


def coefficients(O, n_hi, rho_d, p_d, lum, kabs, kF):
    """kappa_k, alpha_F,k and j_k of the single Cartesian cell from the printed
    step-2 definitions, with the oracle's bin tables (dnu_k, <H>_k and the
    emission factor w_k / (4 pi dx^3 dnu_k)) as inputs."""
    t = O.tables()
    alpha = n_hi * oracle.line_constants(1.0e4)["sigma0"]
    aH = alpha * t["Havg"]
    kap = rho_d * kabs + p_d * aH
    aF = aH + rho_d * kF
    return t["dnu"], kap, aF, lum * t["gem"]


def run_cell(kw, J0, Hx0, Hy0, accept, dt=None):
    O = oracle.Oracle(accept=accept, **kw)
    O.subcycle_on(True)
    s = (J0.reshape(-1, 1, 1), Hx0.reshape(-1, 1, 1), Hy0.reshape(-1, 1, 1))
    J, Hx, Hy, fx, fy, d = O.substep(*s, dt=dt)
    return O, J.ravel(), Hx.ravel(), Hy.ravel(), fx, fy, d, int(O.nsub.ravel()[0])


def _state(nb, seed, scale):
    g = np.random.default_rng(seed)
    J = scale * np.exp(g.normal(0, 0.5, nb))
    f = g.uniform(0, 0.9, nb)
    return J, 0.6 * f * J, -0.7 * f * J


def test_small_change_takes_one_substep_equal_to_the_plain_update():
    # a populated cloud whose every cell changes by less than 10 % in one step:
    # the rule is the plain step-2 update, bit for bit, with frequency step
    c = wl.lognormal_cloud(20, 14, seed=5, L_sun=1e2, Z=1e-4)
    st = wl.populated_state(c, 194, seed=3, J0=1e-9)
    Oa = oracle.Oracle(edges=oracle.freq_grid(), accept=True, **c.kwargs())
    Oa.subcycle_on(True)
    Ob = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
    ra = Oa.substep(*st)
    rb = Ob.substep(*st)
    assert np.all(Oa.nsub == 1)
    for a, b in zip(ra[:5], rb[:5]):
        assert np.array_equal(a, b)
    for k in ("emitted", "absorbed", "outflow", "work", "e_after"):
        assert ra[5][k] == pytest.approx(rb[5][k], rel=1e-13)


@pytest.mark.parametrize("case", ["stiff_absorber", "strong_source", "empty_cell", "destruction"])
def test_single_cell_against_brute_force(case):
    dx = 1e16
    n_hi, rho_d, p_d, lum = 1e3, 0.0, 0.0, 0.0
    J0, Hx0, Hy0 = _state(194, 1, 1e-12)
    if case == "stiff_absorber":      # dust: c dt kappa ~ 50 in one RT step
        rho_d = 1e-18
    elif case == "strong_source":     # emission raises e by ~x10 in one step
        lum = 1e38
    elif case == "empty_cell":        # nothing to start from: the floor decides
        lum, J0, Hx0, Hy0 = 1e20, 0 * J0, 0 * J0, 0 * J0
    elif case == "destruction":       # Lya destruction p_d alpha <H> of a line-core field
        p_d = 1e-3
        core = np.exp(-0.5 * ((np.arange(194) - 96.5) / 6.0) ** 2)
        J0, Hx0, Hy0 = J0 * core, Hx0 * core, Hy0 * core
    kw = one_cell(n_hi, rho_d, p_d, lum, dx=dx)
    O, J, Hx, Hy, fx, fy, d, n = run_cell(kw, J0, Hx0, Hy0, True)
    dnu, kap, aF, js = coefficients(O, n_hi, rho_d, p_d, lum, wl.KAPPA_ABS, wl.KAPPA_F)
    dt = O.dt_cfl
    bJ, bHx, bHy, steps, ax, ay, em, ab = brute_step2(J0, Hx0, Hy0, dnu, kap, aF, js, dt, C_LIGHT)
    assert n == len(steps) > 1  # every case here needs more than one substep
    assert sum(steps) == dt     # the accepted substeps fill the RT step exactly
    np.testing.assert_allclose(J, bJ, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(Hx, bHx, rtol=1e-12, atol=1e-30 * abs(bJ).max() + 1e-300)
    np.testing.assert_allclose(Hy, bHy, rtol=1e-12, atol=1e-30 * abs(bJ).max() + 1e-300)
    fcoef = 4 * math.pi / (C_LIGHT * C_LIGHT * dt)
    assert fx.ravel()[0] == pytest.approx(fcoef * ax, rel=1e-12, abs=1e-300)
    assert fy.ravel()[0] == pytest.approx(fcoef * ay, rel=1e-12, abs=1e-300)
    eunit = 4 * math.pi / C_LIGHT * dx ** 3
    assert d["emitted"] == pytest.approx(eunit * em, rel=1e-12, abs=1e-300)
    assert d["absorbed"] == pytest.approx(eunit * ab, rel=1e-12, abs=1e-300)
    # every accepted substep changed the cell's energy by less than 10 % (+ floor)
    Jb = list(J0)
    for h in steps:
        new = [(Jb[k] + C_LIGHT * h * js[k]) / (1 + C_LIGHT * h * kap[k]) for k in range(194)]
        e0 = sum(dnu[k] * Jb[k] for k in range(194))
        e1 = sum(dnu[k] * new[k] for k in range(194))
        assert abs(e1 - e0) / (e0 + J_FLOOR) < 0.1
        Jb = new


def test_empty_cell_first_substep_is_set_by_the_floor():
    # no absorption: each substep adds c h sum_k dnu_k j_k to e; from e = 0 the
    # first accepted substep is the longest dt / 2^l with c h S < 0.1 J_floor,
    # and the final J is the whole step's emission, however it was split
    dx, lum = 1e16, 1e20
    kw = one_cell(1e3, 0.0, 0.0, lum, dx=dx)
    z = np.zeros(194)
    O, J, Hx, Hy, fx, fy, d, n = run_cell(kw, z, z, z, True)
    dnu, kap, aF, js = coefficients(O, 1e3, 0.0, 0.0, lum, wl.KAPPA_ABS, wl.KAPPA_F)
    dt = O.dt_cfl
    S = float(np.sum(dnu * js))
    l0 = next(l for l in range(41) if C_LIGHT * (dt / 2 ** l) * S < 0.1 * J_FLOOR)
    steps = brute_step2(z, z, z, dnu, kap, aF, js, dt, C_LIGHT)[3]
    assert steps[0] == dt / 2 ** l0 and l0 > 4
    assert n == len(steps)
    np.testing.assert_allclose(J, C_LIGHT * dt * js, rtol=1e-12)


@pytest.mark.parametrize("geometry", [0, 1])
def test_energy_balance_with_the_rule_on(geometry):
    if geometry == 0:
        c = wl.lognormal_cloud(24, 20, seed=8, L_sun=1e7, v_edge_kms=30.0)
    else:
        c = wl.uniform_sphere(24, tau_cl=1e5)
    kw = c.kwargs()
    O = oracle.Oracle(edges=oracle.freq_grid(), accept=True, **kw)
    O.subcycle_on(True)
    st = O.zero_state()
    nmax = 0
    for _ in range(4):
        r = O.substep(*st)
        st = r[:3]
        nmax = max(nmax, int(O.nsub.max()))
        d = r[5]
        scale = max(abs(d["e_after"]), abs(d["emitted"]), 1e-300)
        assert abs(d["residual"]) < 1e-12 * scale
    assert nmax > 1  # the source cells start empty and subcycle


def test_bands_refuse_the_rule():
    z = np.zeros((2, 4, 4))
    with pytest.raises(ValueError):
        oracle.Oracle(nx=4, ny=4, dx=1e16, edges=None, T=1e4, n_hi=0.0, rho_d=0.0, p_d=0.0,
                      ux=0.0, uy=0.0, lum=0.0, freq_step=False, recoil=False,
                      bands=(z + 1e-18, z + 1e-18, z), accept=True)

"""Pins for the oracle's dynamic reduced speed of light (Sec. 2.1, the
dynamic-RSL equation, its f_abs factor, the c_min floor, the c cap and the
-25 % / x4 rate limits).

Each pin is fixed by the limits and scalings the paper derives the rule from,
not by the oracle's own arithmetic:
- free streaming (a_v tau_0 < 1): c_tilde = eps_RSL max(|u|, c_s), linear in
  eps_RSL, the fastest cell deciding wherever it sits;
- optically thick, dust free: c_tilde grows as (a_v tau_0)^(1/3), so x8 in
  n_HI is x2 in c_tilde, and a_v tau_0 ~ 1/T at fixed n_HI (Doppler width
  ~ sqrt(T)) makes x4 in T a factor 4^(-1/3);
- f_abs halves the trapping factor where (a_v tau_0)^(1/3) tau_c = 1 or
  0.6 p_d tau_0 = 1, and removes it where either is large;
- the neutral-gas sound speed scales as sqrt(T) and is about 10 km/s at 10^4 K;
- the RT time step follows c_tilde: dt (c_tilde + |u|_max) is unchanged.
"""
import numpy as np
import pytest

import oracle

KM = 1.0e5
C = 2.99792458e10


def _oracle(n_hi, ux=0.0, uy=0.0, T=1e4, kappa_abs=0.0, rho_d=0.0, p_d=0.0, c_tilde=C,
            temp=None, nx=9, ny=7, dx=3e16):
    z = np.zeros((ny, nx))
    b = lambda a: np.broadcast_to(np.asarray(a, float), (ny, nx))  # noqa: E731
    return oracle.Oracle(nx=nx, ny=ny, dx=dx, edges=oracle.freq_grid(), T=T, n_hi=b(n_hi),
                         rho_d=b(rho_d), p_d=b(p_d), ux=b(ux), uy=b(uy), lum=z,
                         kappa_abs=kappa_abs, c_tilde=c_tilde, gray=True, temp=temp)


def _n_for_tau0(tau0, T=1e4, dx=3e16):
    return tau0 / (oracle.line_constants(T)["sigma0"] * dx)


def test_free_streaming_limit_is_eps_times_fastest_speed():
    g = np.random.default_rng(5)
    ux = g.uniform(-50, 50, (7, 9)) * KM
    uy = g.uniform(-50, 50, (7, 9)) * KM
    umax = np.hypot(ux, uy).max()
    cs = np.full((7, 9), 5.0 * KM)
    for eps in (4.0, 2.5):
        O = _oracle(_n_for_tau0(10.0), ux, uy, c_tilde=eps * umax)
        ct = O.dynamic_ctilde(cs=cs, eps_rsl=eps, ct_min=0.0)
        assert ct == pytest.approx(eps * umax, rel=1e-14)
    # the fastest cell decides wherever it sits; a sound speed above every
    # flow speed takes over
    k = np.unravel_index(np.argmax(np.hypot(ux, uy)), ux.shape)
    perm = np.random.default_rng(6).permutation(63)
    O2 = _oracle(_n_for_tau0(10.0), ux.ravel()[perm].reshape(7, 9),
                 uy.ravel()[perm].reshape(7, 9), c_tilde=4 * umax)
    assert O2.dynamic_ctilde(cs=cs, ct_min=0.0) == pytest.approx(4 * umax, rel=1e-14)
    cs2 = cs.copy()
    cs2[k] = 2 * umax
    O3 = _oracle(_n_for_tau0(10.0), ux, uy, c_tilde=8 * umax)
    assert O3.dynamic_ctilde(cs=cs2, ct_min=0.0) == pytest.approx(8 * umax, rel=1e-14)


def test_thick_dust_free_cube_root_scalings():
    cs = 8.0 * KM
    ref = _oracle(_n_for_tau0(1e7), c_tilde=3e7)
    ct0 = ref.dynamic_ctilde(cs=cs, ct_min=0.0)
    X = ct0 / (4 * cs)
    a_v = oracle.line_constants(1e4)["a_v"]
    assert X == pytest.approx((a_v * 1e7) ** (1.0 / 3.0), rel=1e-13)
    ct8 = _oracle(8 * _n_for_tau0(1e7), c_tilde=3e7).dynamic_ctilde(cs=cs, ct_min=0.0)
    assert ct8 / ct0 == pytest.approx(2.0, rel=1e-13)
    # same n_HI at 4x the temperature (scalar and per-cell field agree)
    n = _n_for_tau0(1e7)
    for kw in ({"T": 4e4}, {"temp": np.full((7, 9), 4e4)}):
        ctT = _oracle(n, c_tilde=3e7, **kw).dynamic_ctilde(cs=cs, ct_min=0.0)
        assert ctT / ct0 == pytest.approx(4.0 ** (-1.0 / 3.0), rel=1e-12)


def test_absorption_factor_terms():
    cs, dx = 8.0 * KM, 3e16
    tau0 = 1e7
    n = _n_for_tau0(tau0)
    ct0 = _oracle(n, c_tilde=3e7).dynamic_ctilde(cs=cs, ct_min=0.0)
    X = ct0 / (4 * cs)
    # continuum absorption depth tau_c = 1 / X halves the trapping factor
    kap = 1.0 / (X * 1e-20 * dx)
    ct = _oracle(n, rho_d=1e-20, kappa_abs=kap, c_tilde=3e7).dynamic_ctilde(cs=cs, ct_min=0.0)
    assert ct / ct0 == pytest.approx(0.5, rel=1e-13)
    # destruction with 0.6 p_d tau_0 = 1 halves it as well
    ct = _oracle(n, p_d=1.0 / (0.6 * tau0), c_tilde=3e7).dynamic_ctilde(cs=cs, ct_min=0.0)
    assert ct / ct0 == pytest.approx(0.5, rel=1e-12)
    # strong absorption or destruction: the factor drops to 1 (max[1, ...])
    for kw in ({"rho_d": 1e-20, "kappa_abs": 10.0 / (1e-20 * dx)}, {"p_d": 1e-3}):
        ct = _oracle(n, c_tilde=4 * cs, **kw).dynamic_ctilde(cs=cs, ct_min=0.0)
        assert ct == pytest.approx(4 * cs, rel=1e-14)


def test_default_sound_speed_of_neutral_gas():
    n = _n_for_tau0(1.0)
    ct1 = _oracle(n, T=1e4, c_tilde=4e6).dynamic_ctilde(ct_min=0.0)
    cs1 = ct1 / 4
    assert 9.5 * KM < cs1 < 11.5 * KM
    ct4 = _oracle(n, T=4e4, c_tilde=8e6).dynamic_ctilde(ct_min=0.0)
    assert ct4 / ct1 == pytest.approx(2.0, rel=1e-13)


def test_floor_cap_and_rate_limits():
    n = _n_for_tau0(1.0)
    # cold static gas: the c_min floor (reached through the -25 % steps)
    O = _oracle(n, T=100.0, c_tilde=1.2e7)
    assert O.dynamic_ctilde(ct_min=1e7) == 1e7
    # faster than light target: capped at c
    O = _oracle(_n_for_tau0(1e8), ux=0.5 * C, c_tilde=C)
    assert O.dynamic_ctilde(cs=1e6) == C
    # from c down to c_min: at most -25 % per update
    O = _oracle(n, T=100.0)
    seen = [C]
    for _ in range(40):
        seen.append(O.dynamic_ctilde(ct_min=1e7))
    steps = np.array(seen[1:]) / np.array(seen[:-1])
    assert np.all(steps >= 0.75 * (1 - 1e-15))
    k = int(np.argmax(np.array(seen) == 1e7))
    np.testing.assert_allclose(seen[1:k], C * 0.75 ** np.arange(1, k), rtol=1e-14)
    assert seen[-1] == 1e7
    # up from 1 km/s: at most x4 per update
    O = _oracle(_n_for_tau0(1e8), ux=100 * KM, c_tilde=1e5)
    a = O.dynamic_ctilde(cs=1e6)
    b = O.dynamic_ctilde(cs=1e6)
    assert a == 4e5 and b == 1.6e6


def test_time_step_follows_ctilde():
    u = 30 * KM
    O = _oracle(_n_for_tau0(1e6), ux=u, c_tilde=C)
    dt0 = O.dt_cfl
    ct = O.dynamic_ctilde(cs=1e6)
    assert ct == 0.75 * C
    assert O.dt_cfl * (ct + u) == pytest.approx(dt0 * (C + u), rel=1e-14)
    O.set_ctilde(3e8)
    assert O.dt_cfl * (3e8 + u) == pytest.approx(dt0 * (C + u), rel=1e-14)


def test_random_field_matches_the_printed_rule():
    # every term on, per-cell temperatures, sound speeds given or defaulted:
    # the printed rule evaluated cell by cell in numpy, with the line constants
    # from their definitions (tau_cell,0 = alpha dx, tau_cell,c = rho_d kappa_abs dx),
    # then the floor, the cap and the rate limits against the previous value.
    # A fast flow lets |u| decide the deciding cell, a slow one c_s.
    KB, MH, ME, QE = 1.380649e-16, 1.67353284e-24, 9.1093837015e-28, 4.803204712570263e-10
    NU0 = C / 1215.67e-8
    nx, ny, dx = 9, 7, 3e16
    g = np.random.default_rng(31)
    T = 10.0 ** g.uniform(3.5, 4.5, (ny, nx))
    n_hi = 10.0 ** g.uniform(-3, 3, (ny, nx))
    rho = 10.0 ** g.uniform(-27, -23, (ny, nx))
    pd = 10.0 ** g.uniform(-8, -3, (ny, nx))
    ux0 = g.uniform(-30, 30, (ny, nx)) * KM
    uy0 = g.uniform(-30, 30, (ny, nx)) * KM
    cs = g.uniform(1, 20, (ny, nx)) * KM
    kabs = 2.682e4
    dnuD = NU0 * np.sqrt(2.0 * KB * T / MH) / C
    a_v = 6.265e8 / (4.0 * np.pi * dnuD)
    sigma0 = np.sqrt(np.pi) * QE * QE * 0.4162 / (ME * C * dnuD)
    tau0 = n_hi * sigma0 * dx
    tauc = rho * kabs * dx
    trap = np.cbrt(a_v * tau0)
    fac = np.maximum(1.0, trap / (1.0 + trap * tauc + 0.6 * pd * tau0))
    cs_neutral = np.sqrt((5.0 / 3.0) * KB * T / (1.22 * MH))
    assert (fac > 1.0).any() and (fac == 1.0).any()
    for scale in (1.0, 0.05):
        ux, uy = scale * ux0, scale * uy0
        speed = np.hypot(ux, uy)
        for c_s, given in ((cs, cs), (cs_neutral, None)):
            term = fac * np.maximum(speed, c_s)
            top = np.unravel_index(np.argmax(term), term.shape)
            assert (speed[top] > c_s[top]) == (scale == 1.0)
            for eps in (4.0, 2.5):
                want = min(max(1e7, eps * term.max()), C)
                assert 1e7 < want < C
                for prev, expect in ((1.2 * want, want), (3.0 * want, 2.25 * want),
                                     (want / 8.0, want / 2.0)):
                    O = _oracle(n_hi, ux, uy, kappa_abs=kabs, rho_d=rho, p_d=pd, c_tilde=prev,
                                temp=T, nx=nx, ny=ny, dx=dx)
                    got = O.dynamic_ctilde(given, eps_rsl=eps, ct_min=1e7)
                    assert got == pytest.approx(expect, rel=1e-12), (scale, eps, prev / want)

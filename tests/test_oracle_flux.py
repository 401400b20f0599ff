"""Pins for the oracle's closure (Levermore M1), the GLF/diffusion interpolation
factor and the face flux (steps A1-A2), against limits and symmetries fixed by
the paper's equations and by the mathematics."""
import math

import numpy as np
import pytest

import oracle


def test_closure_isotropic_and_free_streaming_limits():
    # Sec. 2.1: D ~ I/3 in the diffusive limit, D ~ h (x) h when beam-like
    Dxx, Dxy, Dyy = oracle.closure(0.0, 0.0)
    assert Dxx == pytest.approx(1 / 3, rel=1e-15) and Dyy == pytest.approx(1 / 3, rel=1e-15)
    assert Dxy == 0.0
    for th in np.linspace(0, 2 * math.pi, 13):
        c, s = math.cos(th), math.sin(th)
        Dxx, Dxy, Dyy = oracle.closure(c, s)
        assert Dxx == pytest.approx(c * c, abs=1e-15)
        assert Dxy == pytest.approx(c * s, abs=1e-15)
        assert Dyy == pytest.approx(s * s, abs=1e-15)


def test_closure_rotation_covariance_and_chi_range():
    g = np.random.default_rng(2)
    prev = None
    for f in np.linspace(0, 1, 101):
        # eigenvalue along h is chi(f), rising monotonically from 1/3 to 1
        chi = oracle.closure(f, 0.0)[0]
        assert 1 / 3 - 1e-15 <= chi <= 1 + 1e-15
        if prev is not None:
            assert chi >= prev
        prev = chi
    for _ in range(200):
        f = g.uniform(0, 1)
        th, rot = g.uniform(0, 2 * math.pi, 2)
        fx, fy = f * math.cos(th), f * math.sin(th)
        D = np.array(oracle.closure(fx, fy))
        D = np.array([[D[0], D[1]], [D[1], D[2]]])
        R = np.array([[math.cos(rot), -math.sin(rot)], [math.sin(rot), math.cos(rot)]])
        fr = R @ np.array([fx, fy])
        Dr = np.array(oracle.closure(fr[0], fr[1]))
        Dr = np.array([[Dr[0], Dr[1]], [Dr[1], Dr[2]]])
        np.testing.assert_allclose(Dr, R @ D @ R.T, atol=1e-14)


def test_eps_limits():
    # eps = 1 when tau -> 0, eps ~ 1/tau when tau >> 1 (Sec. 2.1)
    assert oracle.eps(0.0) == 1.0
    for tau in (1e4, 1e6, 1e8, 1e12):
        assert oracle.eps(tau) * tau == pytest.approx(1.0, rel=2.0 / tau)
    taus = np.logspace(-6, 8, 300)
    e = np.array([oracle.eps(t) for t in taus])
    assert np.all(np.diff(e) < 0) and np.all(e > 0) and np.all(e <= 1)


def test_face_flux_uniform_state():
    # no gradients, isotropic: no energy flux, H_n flux = K_nn = J/3
    out = oracle.face_flux([2, 2, 2, 2], [0, 0, 0, 0], [0, 0, 0, 0], 3.0, 3.0, 0, 0, 1.0)
    assert out[0] == 0.0
    assert out[1] == pytest.approx(2 / 3, rel=1e-15)
    assert out[2] == 0.0


def test_face_flux_free_streaming_beam():
    # f = 1 along the normal in vacuum: the GLF flux is exact upwinding, F_J = J
    out = oracle.face_flux([1, 1, 1, 1], [1, 1, 1, 1], [0, 0, 0, 0], 0, 0, 0, 0, 1.0)
    np.testing.assert_allclose(out, [1.0, 1.0, 0.0], atol=1e-15)
    # beam front entering empty cells
    out = oracle.face_flux([1, 1, 0, 0], [1, 1, 0, 0], [0, 0, 0, 0], 0, 0, 0, 0, 1.0)
    assert out[0] == pytest.approx(1.0, rel=1e-15)
    # oblique beam: energy flux = normal component of H
    c, s = math.cos(0.3), math.sin(0.3)
    out = oracle.face_flux([1, 1, 1, 1], [c] * 4, [s] * 4, 0, 0, 0, 0, 1.0)
    np.testing.assert_allclose(out, [c, c * c, c * s], atol=1e-15)


def test_face_flux_thick_limit_is_diffusion():
    # tau >> 1: F_J -> -(J_{i+1} - J_i) / (3 tau) (discretised -grad J / 3 alpha_F)
    dx = 2.0
    for tau in (1e3, 1e6, 1e9):
        aF = tau / dx
        out = oracle.face_flux([1, 2, 3, 4], [0] * 4, [0] * 4, aF, aF, 0, 0, dx)
        assert out[0] * 3 * tau == pytest.approx(-1.0, rel=2.0 / tau)
        # K flux is central: (K^L + K^R)/2 = J_face / 3
        assert out[1] == pytest.approx(2.5 / 3, rel=1e-14)


def test_face_flux_mirror_symmetry():
    g = np.random.default_rng(11)
    for _ in range(300):
        J = g.uniform(0.1, 2, 4)
        f = g.uniform(-0.7, 0.7, (2, 4))
        Hn, Ht = J * f[0], J * f[1]
        aF0, aF1 = g.uniform(0, 5, 2)
        u0, u1 = g.uniform(-1e8, 1e8, 2)
        a = oracle.face_flux(J, Hn, Ht, aF0, aF1, u0, u1, 1.0)
        # reflect the normal axis: reverse cells, negate normal components
        b = oracle.face_flux(J[::-1], -Hn[::-1], Ht[::-1], aF1, aF0, -u1, -u0, 1.0)
        np.testing.assert_allclose([b[0], b[1], b[2]], [-a[0], a[1], -a[2]], rtol=1e-13,
                                   atol=1e-15 * np.abs(a).max())


def test_face_flux_advection_upwind():
    c = 2.99792458e10
    u = 0.01 * c
    # uniform isotropic gas moving along +n: F_J = u J / c, F_n = K_nn + u H_n / c
    out = oracle.face_flux([3] * 4, [0] * 4, [0] * 4, 1.0, 1.0, u, u, 1.0)
    assert out[0] == pytest.approx(0.03, rel=1e-14)
    assert out[1] == pytest.approx(1.0, rel=1e-14)
    # donor is the upwind side: J = [1,1,5,5] step, u > 0 takes the left state
    out_p = oracle.face_flux([1, 1, 5, 5], [0] * 4, [0] * 4, 1e9, 1e9, u, u, 1.0)
    out_m = oracle.face_flux([1, 1, 5, 5], [0] * 4, [0] * 4, 1e9, 1e9, -u, -u, 1.0)
    diff0 = oracle.face_flux([1, 1, 5, 5], [0] * 4, [0] * 4, 1e9, 1e9, 0, 0, 1.0)[0]
    assert out_p[0] - diff0 == pytest.approx(0.01 * 1, rel=1e-6)
    assert out_m[0] - diff0 == pytest.approx(-0.01 * 5, rel=1e-6)

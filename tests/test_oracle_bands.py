"""Pins for the oracle's broad bands (Sec. 3: stellar and IR bands solved with
the M1 moment equations of Sec. 2.1 per band, without frequency-derivative
terms; per-[band][cell] flux and absorption opacities and emissivity).

- A band given the opacities and emission of the gray Lya group (alpha_F =
  alpha eta + rho_d kappa_F, kappa = rho_d kappa_abs + p_d alpha eta,
  j = L / (4 pi V)) is that group, bit for bit: the band inputs replace the
  group's opacity formulas and nothing else (the gray group is pinned by the
  substep pins).
- A uniform medium with emission j and absorption kappa relaxes to the
  steady state J = j / kappa of 1/c dJ/dt = j - kappa J, with H = 0.
- Bands do not couple: a run with several bands equals one run per band.
- Thin uniform sphere with a gray band (axisymmetric grid): the force
  multiplier tends to tau / 4 with tau = alpha_F R (Sec. 4.1, Test 1, thin
  limit, with eta = 1 for a band).
- Energy bookkeeping closes to round-off with every term on.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl

C = 2.99792458e10


def _gray_to_bands(c, O):
    """Band inputs equal to the gray group of cloud c (Cartesian cells)."""
    alpha = c.n_hi * oracle.line_constants(c.T)["sigma0"]
    aH = alpha * O.eta
    kap = c.rho_d * c.kappa_abs + c.p_d * aH
    aF = aH + c.rho_d * c.kappa_F
    gem = 1.0 / ((4.0 * math.pi) * ((c.dx * c.dx) * c.dx))
    js = c.lum * gem
    return aF[None], kap[None], js[None]


def test_band_reduces_to_gray_group():
    c = wl.lognormal_cloud(21, 17, seed=41, Z=0.5, p_d=1e-6, v_edge_kms=300.0)
    c.gray = True
    for bc in ((0, 0, 0, 0), (1, 1, 0, 1)):
        c.bc = bc
        G = oracle.Oracle(edges=oracle.freq_grid(), **c.kwargs())
        B = oracle.Oracle.for_bands(nx=c.nx, ny=c.ny, dx=c.dx, ux=c.ux, uy=c.uy, bc=bc,
                                    **dict(zip(("alpha_F", "kappa", "emissivity"),
                                                           _gray_to_bands(c, G))))
        assert B.nb == 1 and B.dt_cfl == G.dt_cfl
        g = np.random.default_rng(42)
        J = 1e-3 * np.exp(g.normal(0, 1, (1, c.ny, c.nx)))
        st = (J, 0.4 * J * g.uniform(-1, 1, J.shape), 0.4 * J * g.uniform(-1, 1, J.shape))
        (rg, dg), (rb, db) = G.run(6, st), B.run(6, st)
        for a, b in zip(rg, rb):
            np.testing.assert_array_equal(a, b)
        for k in ("emitted", "absorbed", "outflow", "work", "e_after"):
            assert dg[-1][k] == db[-1][k]


def test_uniform_medium_relaxes_to_j_over_kappa():
    n, dx = 6, 1e17
    aF, kap, j = 3e-17, 2e-17, 5e-24
    B = oracle.Oracle.for_bands(nx=n, ny=n, dx=dx, alpha_F=np.full((1, n, n), aF),
                                kappa=np.full((1, n, n), kap), emissivity=np.full((1, n, n), j))
    (J, Hx, Hy, fx, fy), d = B.run(400)
    np.testing.assert_allclose(J, j / kap, rtol=1e-12)
    assert np.all(Hx == 0.0) and np.all(Hy == 0.0) and np.all(fx == 0.0)
    # implicit step 2 on a uniform field: J_n = (J_{n-1} + ct dt j) / (1 + ct dt kappa)
    (J1, _, _, _, _), _ = B.run(1)
    cdt = C * B.dt_cfl
    np.testing.assert_allclose(J1, cdt * j / (1.0 + cdt * kap), rtol=1e-15)


def test_bands_are_independent():
    nx, ny, nb = 19, 14, 3
    g = np.random.default_rng(43)
    dx = 3e16
    tau = 10.0 ** g.uniform(-2, 2, (nb, ny, nx))
    aF = tau / dx
    kap = aF * g.uniform(0.1, 1.0, aF.shape)
    j = np.zeros((nb, ny, nx))
    j[:, 6:8, 9:11] = 1e-20 * np.array([1.0, 3.0, 0.5])[:, None, None]
    u = wl.radial_velocity(nx, ny, dx, 200.0 * wl.KM, nx * dx)
    kw = dict(nx=nx, ny=ny, dx=dx, ux=u[0], uy=u[1], bc=(1, 1, 1, 1))
    all_ = oracle.Oracle.for_bands(alpha_F=aF, kappa=kap, emissivity=j, **kw)
    (J, Hx, Hy, fx, fy), d = all_.run(8)
    assert all(abs(x["residual"]) <= 1e-13 * x["e_after"] for x in d[1:])
    fsum = np.zeros_like(fx)
    for b in range(nb):
        one = oracle.Oracle.for_bands(alpha_F=aF[b:b + 1], kappa=kap[b:b + 1],
                                      emissivity=j[b:b + 1], **kw)
        assert one.dt_cfl == all_.dt_cfl
        (Jb, Hxb, Hyb, fxb, fyb), _ = one.run(8)
        np.testing.assert_array_equal(J[b], Jb[0])
        np.testing.assert_array_equal(Hx[b], Hxb[0])
        np.testing.assert_array_equal(Hy[b], Hyb[0])
        fsum += fxb
    np.testing.assert_allclose(fx, fsum, rtol=1e-12, atol=1e-12 * np.abs(fsum).max())


def test_thin_sphere_band_force_multiplier():
    n, tau = 32, 0.1
    s = wl.uniform_sphere(n, tau_cl=tau, gray=True)
    R = s.meta["R_cl"]
    inside = s.n_hi > 0
    aF = np.where(inside, tau / R, 0.0)[None]
    j = np.where(inside, 1e-22, 0.0)[None]
    B = oracle.Oracle.for_bands(nx=n, ny=n, dx=s.dx, alpha_F=aF, kappa=np.zeros_like(aF),
                                emissivity=j, geometry=1, bc=(0, 1, 0, 1))
    _, d = B.run(int(60 * R / s.dx))
    # L of the half-space Z > 0: 4 pi j over the ring volumes pi (2i + 1) dx^3
    ring = math.pi * (2.0 * np.arange(n) + 1.0) * s.dx ** 3
    L = (4.0 * math.pi * j[0] * ring[None, :]).sum()
    mf = d[-1]["force_abs"] / (L / C)
    assert abs(mf / (tau / 4.0) - 1.0) < 0.02
    assert abs(d[-1]["force_radial"] / d[-1]["force_abs"] - 1.0) < 2e-3
    assert abs(d[-1]["residual"]) < 1e-12 * d[-1]["e_after"]


def test_invalid_band_problems():
    z = np.zeros((1, 4, 4))
    with pytest.raises(ValueError):
        oracle.Oracle(nx=4, ny=4, dx=1e16, edges=None, T=1e4, n_hi=0, rho_d=0, p_d=0, ux=0,
                      uy=0, lum=0, gray=True, bands=(z, z, z))


def test_stellar_band_inputs():
    # the seven-band recipe: absorption never exceeds the flux opacity (kappa_abs
    # <= kappa_F in the dust table, gas absorption counted in both), the six
    # stellar bands together carry the cloud's luminosity, and the IR band's
    # emissivity is the dust's rho_d kappa_IR sigma T_d^4 / pi
    c = wl.lognormal_cloud(24, 20, seed=181, Z=0.3)
    aF, ka, je = wl.stellar_bands(c, T_dust=25.0)
    assert aF.shape == ka.shape == je.shape == (7, 20, 24)
    assert np.all(ka <= aF * (1 + 1e-15)) and np.all(ka >= 0) and np.all(je >= 0)
    V = c.dx ** 3
    L6 = (4.0 * math.pi * je[1:] * V).sum()
    assert L6 == pytest.approx(c.lum.sum(), rel=1e-12)
    np.testing.assert_allclose(je[0], c.rho_d * wl.KAPPA_IR * wl.SIGMA_SB * 25.0 ** 4 / math.pi,
                               rtol=1e-15)
    # EUV1 is absorbed by neutral gas far more strongly than the optical band
    assert np.all(ka[4] > 100 * ka[1])

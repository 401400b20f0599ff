"""Pins for the oracle's axisymmetric (R, Z) substep (Sec. 2.1 finite volumes in
cylindrical coordinates, Sec. 4.1 test set-up: reflecting axis, mirrored
midplane, outflow outer edges).

Each pin is fixed by the physics or the mathematics, not by the oracle:
- the thin-sphere force multiplier M_F = tau_cl eta / 4 (Sec. 4.1, Test 1,
  the optically thin limit): in a steady state div F equals the emissivity,
  so for uniform emission in a sphere F = L r / (4 pi R^3) whatever the
  closure, and the force integral is fixed (a Cartesian slab would give
  tau eta / 3, a dropped hoop term or a wrong face area moves it too);
- M_F = M_F,radial in a spherically symmetric cloud (Sec. 4);
- a uniform isotropic field is steady (the R-face flux difference of K_RR
  balances the hoop term K_phiphi <1/R>);
- the work term of a uniform isotropic field in a Hubble flow u = a r equals
  (e/c) a c_tilde dt V, the trace of grad u being 3a (hoop part included);
- photon bookkeeping closes to round-off with every term active.
"""
import math

import numpy as np

import oracle
import workloads as wl

C = 2.99792458e10


def _gray_cyl(n, n_hi, lum=None, ux=None, uy=None, dx=1e16):
    z = np.zeros((n, n))
    return oracle.Oracle(nx=n, ny=n, dx=dx, edges=oracle.freq_grid(), T=1e4,
                         n_hi=np.broadcast_to(n_hi, (n, n)), rho_d=z, p_d=z,
                         ux=z if ux is None else ux, uy=z if uy is None else uy,
                         lum=z if lum is None else lum, gray=True, geometry=1)


def _thin_sphere_mf(n, tau):
    cl = wl.uniform_sphere(n, tau_cl=tau, gray=True)
    O = oracle.Oracle(edges=oracle.freq_grid(), **cl.kwargs())
    R_cl = cl.meta["R_cl"]
    # optical depth with the oracle's own line-centre cross-section
    tau_eff = float(cl.n_hi.max()) * oracle.line_constants(cl.T)["sigma0"] * R_cl
    steps = int(60 * R_cl / cl.dx)  # about 12 light-crossing times of the cloud
    _, diags = O.run(steps)
    d = diags[-1]
    L = cl.L_total
    return d["force_abs"] / (L / C), d["force_radial"] / (L / C), tau_eff * O.eta / 4.0, d


def test_thin_sphere_force_multiplier():
    mf32, mr32, pred, d = _thin_sphere_mf(32, 0.1)
    assert abs(mf32 / pred - 1.0) < 0.02
    # spherical symmetry: the force is radial
    assert abs(mr32 / mf32 - 1.0) < 1e-3
    # steady: the bookkeeping residual is round-off
    assert abs(d["residual"]) < 1e-12 * d["e_after"]
    mf64, _, _, _ = _thin_sphere_mf(64, 0.1)
    # first-order convergence toward the exact limit
    assert abs(mf64 / pred - 1.0) < 0.5 * abs(mf32 / pred - 1.0)


def test_uniform_isotropic_field_is_steady():
    n = 12
    O = _gray_cyl(n, 0.0)
    J = np.full((1, n, n), 2.5)
    Hx = np.zeros_like(J)
    Hy = np.zeros_like(J)
    for _ in range(5):
        J, Hx, Hy, fx, fy, d = O.substep(J, Hx, Hy)
        assert np.max(np.abs(Hx)) < 1e-14 * 2.5
        assert np.max(np.abs(Hy)) == 0.0
    np.testing.assert_allclose(J, 2.5, rtol=1e-13)


def test_hubble_flow_work_term():
    # J uniform inside an m x m block away from the outer edges (where the
    # copied ghosts break linearity), zero outside; H = 0; u = a (R, Z)
    n, m, dx, a = 16, 10, 1e16, 1e-9
    c = (np.arange(n) + 0.5) * dx
    R, Z = np.meshgrid(c, c)
    O = _gray_cyl(n, 0.0, ux=a * R, uy=a * Z, dx=dx)
    J0 = 1.7
    J = np.zeros((1, n, n))
    J[0, :m, :m] = J0
    H = np.zeros_like(J)
    dt = O.dt_cfl
    _, _, _, _, _, d = O.substep(J, H, H, dt)
    V = math.pi * (m * dx) ** 2 * (m * dx)   # 2 pi int_0^{m dx} R dR dZ
    e = (4.0 * math.pi / C) * J0 * V
    expect = e * a * (C * dt) / C
    assert abs(d["work"] / expect - 1.0) < 1e-12


def test_energy_bookkeeping_cylindrical_full_physics(paper_edges):
    c = wl.lognormal_cloud(20, 16, seed=11, Z=0.5, p_d=1e-6, v_edge_kms=300.0)
    c.geometry = 1
    O = oracle.Oracle(edges=paper_edges, **c.kwargs())
    _, diags = O.run(40)
    for d in diags[1:]:
        assert abs(d["residual"]) <= 1e-13 * d["e_after"]
        assert d["absorbed"] > 0 and d["work"] != 0
    assert diags[-1]["outflow"] > 0


def test_cone_density_field():
    # Sec. 4.2 (Test 6) set-up: the cone axis is near tau_cone, the midplane
    # shell near tau_cl, the core scaled by eps_core, vacuum outside R_cl
    cl = wl.cone_cloud(64)
    s0 = wl.SIGMA0_1E4K
    R_cl = cl.meta["R_cl"]
    n_axis = cl.n_hi[-8, 0]      # mu ~ 1, r ~ R_cl: shell inside the cone
    n_mid = cl.n_hi[0, 45]       # mu ~ 0: shell outside the cone
    assert abs(n_axis * s0 * R_cl / 1e5 - 1.0) < 1e-3
    assert abs(n_mid * s0 * R_cl / 1e8 - 1.0) < 1e-3
    assert cl.n_hi[0, 0] * s0 * R_cl < 1e8 * 2e-4
    assert cl.n_hi[-1, -1] == 0.0
    # emission only inside 0.5 R_cl
    c = (np.arange(64) + 0.5) * cl.dx
    Rg, Zg = np.meshgrid(c, c)
    assert np.all(cl.lum[np.hypot(Rg, Zg) > 0.5 * R_cl] == 0.0)

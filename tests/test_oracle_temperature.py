"""Pins for a per-cell gas temperature (App. A: <H>_k, the Doppler width, a_v
and sigma0 at each cell's own T; the recoil factor h/(k_B T) of step 3).

- A uniform temperature field equal to the scalar T reproduces the scalar-T
  substep bit for bit (Cartesian and axisymmetric, 194 bins, recoil, flow).
- Two cells at different temperatures starting from the same isotropic state
  exchange nothing in their first substep (equal states give zero net face
  fluxes), so each must equal a one-cell run at its own temperature: this
  pins every per-cell table and the per-cell frequency step to the
  single-temperature A0 path, itself pinned against quadrature and printed
  constants (test_oracle_tables).
"""
import numpy as np

import oracle
import workloads as wl


def test_uniform_field_equals_scalar_temperature(paper_edges):
    for geometry in (0, 1):
        c = wl.lognormal_cloud(13, 9, seed=41, v_edge_kms=80.0, Z=0.3, p_d=1e-5)
        c.geometry = geometry
        kw = c.kwargs()
        A = oracle.Oracle(edges=paper_edges, **kw)
        kw2 = dict(kw, temp=np.full((9, 13), c.T))
        B = oracle.Oracle(edges=paper_edges, **kw2)
        sa, da = A.run(3)
        sb, db = B.run(3)
        for a, b in zip(sa, sb):
            np.testing.assert_array_equal(a, b)
        assert da[-1] == db[-1]


def test_cells_at_two_temperatures_match_one_cell_runs(paper_edges):
    nb = paper_edges.size - 1
    T = np.array([[300.0, 2.0e4]])
    g = np.random.default_rng(5)
    spec = np.exp(-0.5 * ((np.arange(nb) - 97) / 6.0) ** 2) + 1e-3
    J = np.repeat(spec[:, None, None], 2, axis=2) * 1e-9
    H = np.zeros_like(J)
    common = dict(ny=1, dx=3e15, n_hi=10.0, rho_d=0.0, p_d=0.0, ux=0.0, uy=0.0, lum=0.0,
                  recoil=True)
    two = oracle.Oracle(nx=2, edges=paper_edges, T=1e4, temp=T, **common)
    dt = two.dt_cfl
    Jo, Hxo, Hyo, _, _, _ = two.substep(J, H, H, dt)
    for i in range(2):
        one = oracle.Oracle(nx=1, edges=paper_edges, T=T[0, i], **common)
        Ji, Hxi, Hyi, _, _, _ = one.substep(J[:, :, i:i + 1], H[:, :, :1], H[:, :, :1], dt)
        np.testing.assert_array_equal(Jo[:, :, i:i + 1], Ji)
    # the two temperatures redistribute differently (recoil and widths)
    assert not np.allclose(Jo[:, 0, 0], Jo[:, 0, 1], rtol=1e-6, atol=0.0)
    # photon number per cell is conserved by step 3 (no sources or sinks)
    tab = oracle.bin_tables(paper_edges, 1e4)
    for i in range(2):
        n0 = (tab["dnu"] * J[:, 0, i]).sum()
        n1 = (tab["dnu"] * Jo[:, 0, i]).sum()
        assert abs(n1 / n0 - 1.0) < 1e-12


def test_two_phase_temperature_field_is_seeded():
    a = wl.two_phase_temperature(32, 16, seed=3)
    b = wl.two_phase_temperature(32, 16, seed=3)
    np.testing.assert_array_equal(a, b)
    assert 100.0 <= a.min() and a.max() <= 1e4
    assert abs((a > 1000.0).mean() - 0.5) < 0.15

"""Pins for the emergent spectrum (the escaping energy per bin and outer face,
Sec. 4's emergent spectra and f_esc): it is the face-by-face split of the
outflow term of the photon bookkeeping, so it must sum to that term; a
mirror-symmetric problem gives mirror-equal spectra on opposite faces; an
outgoing beam leaves only through its own face."""
import numpy as np

import oracle
import workloads as wl


def test_spectrum_sums_to_outflow(paper_edges):
    for geometry, bc in ((0, (0, 0, 0, 0)), (0, (1, 1, 1, 1)), (1, (0, 1, 0, 1))):
        c = wl.lognormal_cloud(14, 11, seed=71, v_edge_kms=50.0, Z=0.2)
        c.geometry, c.bc = geometry, bc
        O = oracle.Oracle(edges=paper_edges, **c.kwargs())
        O.spectrum_on()
        g = np.random.default_rng(72)
        J = 1e-12 * np.exp(g.normal(0, 1, (O.nb, 11, 14)))
        Hx = 0.5 * J * g.uniform(-1, 1, J.shape)
        Hy = 0.5 * J * g.uniform(-1, 1, J.shape)
        for _ in range(3):
            J, Hx, Hy, _, _, d = O.substep(J, Hx, Hy)
            s = O.spectrum
            assert s.shape == (O.nb, O.n_faces())
            assert abs(s.sum() - d["outflow"]) <= 1e-12 * np.abs(s).sum()


def test_mirror_symmetric_problem_has_mirror_spectra(paper_edges):
    n = 12
    c = wl.uniform_gray(n, n)
    O = oracle.Oracle(edges=paper_edges, **c.kwargs())
    O.spectrum_on()
    J, Hx, Hy = O.zero_state()
    for _ in range(30):
        J, Hx, Hy, _, _, _ = O.substep(J, Hx, Hy)
    s = O.spectrum[0]
    xm, xp, ym, yp = s[:n], s[n:2 * n], s[2 * n:3 * n], s[3 * n:]
    scale = np.abs(s).max()
    assert scale > 0
    np.testing.assert_allclose(xm, xp, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(ym, yp, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(xm, ym, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(xm, xm[::-1], rtol=0, atol=1e-12 * scale)


def test_outgoing_beam_leaves_through_its_face(paper_edges):
    nx, ny = 8, 3
    z = np.zeros((ny, nx))
    O = oracle.Oracle(nx=nx, ny=ny, dx=1e15, edges=paper_edges, T=1e4, n_hi=z, rho_d=z, p_d=z,
                      ux=z, uy=z, lum=z, gray=True, bc=(1, 1, 0, 0))
    O.spectrum_on()
    J = np.ones((1, ny, nx))
    J, Hx, Hy, _, _, d = O.substep(J, J.copy(), np.zeros_like(J))
    s = O.spectrum[0]
    assert np.all(s[ny:2 * ny] > 0)                       # x+ faces carry the beam
    np.testing.assert_array_equal(s[:ny], 0.0)            # x-: (H_R - J_R)/2 = 0
    np.testing.assert_array_equal(s[2 * ny:], 0.0)        # y faces: no normal flux
    assert abs(s.sum() - d["outflow"]) <= 1e-14 * s.sum()

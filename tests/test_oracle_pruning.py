"""Pins for active-bin pruning in the oracle (Sec. 2.2: only bins holding more
than a fraction, 1e-10 in the paper, of the domain's Lya energy are advected;
the others skip step 1 and still take steps 2 and 3).

- A cut below every bin's share is the unpruned substep, bit for bit.
- In vacuum, without sources or a frequency step, a pruned bin comes out of
  the substep exactly as it went in (steps 2 and 3 leave it alone there),
  while an active bin streams: its outflow is nonzero.
- The cut is strict and relative to the total: shares of 2e-10 stay active
  and 5e-11 are pruned at 1e-10, whatever the overall scale.
- The energy bookkeeping still closes to round-off.
"""
import numpy as np

import oracle
import workloads as wl

EDGES = oracle.freq_grid()


def _state(nb, ny, nx, seed, share=None):
    g = np.random.default_rng(seed)
    J = np.exp(g.normal(0, 0.5, (nb, ny, nx)))
    Hx = 0.5 * J * g.uniform(-1, 1, J.shape)
    Hy = 0.5 * J * g.uniform(-1, 1, J.shape)
    if share is not None:  # bins scaled to a given share of the total energy
        for k, f in share.items():
            for a in (J, Hx, Hy):
                a[k] *= f
    return J, Hx, Hy


def test_cut_below_every_share_is_unpruned():
    c = wl.lognormal_cloud(19, 13, seed=161, v_edge_kms=80.0, Z=0.3, p_d=1e-7)
    st = _state(194, 13, 19, 162)
    a = oracle.Oracle(edges=EDGES, **c.kwargs())
    b = oracle.Oracle(edges=EDGES, prune=1e-300, **c.kwargs())
    (ra, da), (rb, db) = a.run(2, st), b.run(2, st)
    for x, y in zip(ra, rb):
        np.testing.assert_array_equal(x, y)
    assert da[-1]["outflow"] == db[-1]["outflow"]


def test_pruned_bins_are_not_advected():
    nx, ny = 16, 12
    z = np.zeros((ny, nx))
    kw = dict(nx=nx, ny=ny, dx=1e16, edges=EDGES, T=1e4, n_hi=z, rho_d=z, p_d=z, ux=z, uy=z,
              lum=z, freq_step=False, bc=(1, 1, 1, 1))
    tiny = {k: 1e-14 for k in range(0, 194, 3)}
    J, Hx, Hy = _state(194, ny, nx, 163, share=tiny)
    O = oracle.Oracle(prune=1e-10, **kw)
    O.spectrum_on()
    Jo, Hxo, Hyo, _, _, d = O.substep(J, Hx, Hy)
    pruned = sorted(tiny)
    active = [k for k in range(194) if k not in tiny]
    for k in pruned:
        np.testing.assert_array_equal(Jo[k], J[k])
        np.testing.assert_array_equal(Hxo[k], Hx[k])
        np.testing.assert_array_equal(Hyo[k], Hy[k])
        assert not np.any(O.spectrum[k])
    assert all(not np.array_equal(Jo[k], J[k]) for k in active)
    assert np.all(O.spectrum[active].sum(axis=1) > 0)
    assert abs(d["residual"]) <= 1e-13 * d["e_before"]
    # without pruning the same bins stream too
    Jo2, _, _, _, _, _ = oracle.Oracle(**kw).substep(J, Hx, Hy)
    assert all(not np.array_equal(Jo2[k], J[k]) for k in pruned)


def test_cut_is_strict_and_relative():
    nx, ny = 10, 8
    z = np.zeros((ny, nx))
    kw = dict(nx=nx, ny=ny, dx=1e16, edges=EDGES, T=1e4, n_hi=z, rho_d=z, p_d=z, ux=z, uy=z,
              lum=z, freq_step=False, bc=(1, 1, 1, 1))
    dnu = oracle.Oracle(**kw).tables()["dnu"]
    for scale in (1.0, 1e-30, 1e25):
        # uniform J per bin; bin 5 at a share 2e-10 of the total, bin 9 at 5e-11
        base = np.ones(194)
        E = base * dnu
        tot_rest = E.sum() - E[5] - E[9]
        base[5] = 2e-10 * tot_rest / (1 - 2.5e-10) / dnu[5]
        base[9] = 5e-11 * tot_rest / (1 - 2.5e-10) / dnu[9]
        J = scale * np.broadcast_to(base[:, None, None], (194, ny, nx)).copy()
        J[:, 3:5, 4:6] *= 2.0  # a bump, so that an advected bin changes
        share = (J.sum(axis=(1, 2)) * dnu) / (J.sum(axis=(1, 2)) * dnu).sum()
        assert 1e-10 < share[5] < 3e-10 and 3e-11 < share[9] < 1e-10
        H = np.zeros_like(J)
        Jo, _, _, _, _, _ = oracle.Oracle(prune=1e-10, **kw).substep(J, H, H)
        assert not np.array_equal(Jo[5], J[5])
        np.testing.assert_array_equal(Jo[9], J[9])


def test_bookkeeping_closes_with_pruning():
    c = wl.lognormal_cloud(20, 16, seed=164, v_edge_kms=200.0, Z=0.5, p_d=1e-6)
    O = oracle.Oracle(edges=EDGES, prune=1e-10, **c.kwargs())
    st = _state(194, 16, 20, 165, share={k: 1e-13 for k in range(0, 194, 2)})
    (_, _, _, _, _), diags = O.run(6, st)
    for d in diags:
        assert abs(d["residual"]) <= 1e-13 * max(d["e_after"], d["e_before"])

"""GPU parity under a per-cell gas temperature (App. A: <H>_k, Doppler width, a_v
and sigma0 at each cell's own T; the recoil factor h/(k_B T) per cell), with
the bars of test_gpu_parity: bit-exact for LYM1_FP64_DET, 1e-10 for LYM1_FP64,
1e-4 per element plus the n u S_n floor for the mixed policies."""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, close, fw_of, random_state, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


def warm_cold_cloud(nx, ny, seed, geometry=0):
    c = wl.lognormal_cloud(nx, ny, seed=seed, v_edge_kms=60.0, Z=0.1, p_d=1e-7)
    c.temp = wl.two_phase_temperature(nx, ny, seed + 100, T_cold=80.0, T_hot=2e4)
    c.geometry = geometry
    return c


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_two_phase_temperature_194_bins(L, edges, precision):
    c = warm_cold_cloud(45, 38, seed=51)
    st = random_state(194, 38, 45, 52)
    got, ref, dg, diags = run_both(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))
    assert dg["e_tot"] == pytest.approx(diags[-1]["e_after"], rel=max(TOL[precision], 1e-12))


@pytest.mark.parametrize("precision", [0, 3])
def test_two_phase_temperature_axisymmetric(L, edges, precision):
    c = warm_cold_cloud(37, 29, seed=53, geometry=1)
    c.bc = (0, 1, 0, 1)
    st = random_state(194, 29, 37, 54)
    got, ref, _, _ = run_both(L, c, edges, precision, 3, st)
    check_outputs(got, ref, TOL[precision], 3, st, fw_of(c, edges))


@pytest.mark.parametrize("precision", [0, 3])
def test_uniform_field_equals_scalar_temperature(L, edges, precision):
    c = wl.lognormal_cloud(40, 24, seed=55, v_edge_kms=40.0)
    st = random_state(194, 24, 40, 56)
    a = L.from_cloud(c, precision=precision, edges=edges)
    c.temp = np.full((24, 40), c.T)
    b = L.from_cloud(c, precision=precision, edges=edges)
    for x in (a, b):
        x.set_state(*st)
        x.substeps(3)
    # bit for bit in FP64_DET; FP32 forms the recoil factor per cell in FP32
    # (one rounding more than the per-bin table), so the mixed bar applies
    check_outputs(a.get_state() + a.force(), b.get_state() + b.force(), TOL[precision], 3, st, fw_of(c, edges))
    a.destroy()
    b.destroy()


def test_gray_group_with_temperature_field(L, edges):
    c = wl.uniform_gray(40, 28)
    c.temp = wl.two_phase_temperature(40, 28, seed=57)
    got, ref, _, _ = run_both(L, c, edges, 0, 20)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 0.0, n)


def test_batches_and_invalid_temperatures(L, edges):
    clouds = [warm_cold_cloud(40, 24, seed=58), warm_cold_cloud(17, 33, seed=59)]
    solo = []
    for c in clouds:
        x = L.from_cloud(c, precision="mixed_fast", edges=edges)
        for _ in range(4):
            x.substeps(1)
        solo.append(x.get_state())
        x.destroy()
    ctxs = [L.from_cloud(c, precision="mixed_fast", edges=edges) for c in clouds]
    b = L.Batch(ctxs)
    b.substeps(4)
    b.destroy()
    for x, s in zip(ctxs, solo):
        for u, w in zip(x.get_state(), s):
            np.testing.assert_array_equal(u, w)
    plain = L.from_cloud(wl.lognormal_cloud(16, 16, seed=60), precision="mixed_fast", edges=edges)
    with pytest.raises(L.Lym1Error) as e:
        L.Batch([plain, ctxs[0]])
    assert e.value.status == L.EINVAL
    plain.destroy()
    for x in ctxs:
        x.destroy()
    bad = warm_cold_cloud(8, 8, seed=61)
    bad.temp[3, 3] = -5.0
    with pytest.raises(L.Lym1Error) as e:
        L.from_cloud(bad, precision="mixed_fast", edges=edges)
    assert e.value.status == L.EINVAL

"""New gas temperatures on the GPU (lym1_set_temperature: the per-cell tables of
App. A and Sec. 2.1 rebuilt by a device kernel).  After a change from one
two-phase field to another, the substeps match the oracle run at the new
temperatures (1e-10 relative in FP64: the device's exp / erf / erfc differ from
the host's in the last bits, so FP64_DET is not bit-exact here; 1e-4 plus the
n u S_n floor for the mixed policies), and a context updated on the device
agrees with one whose tables were built on the host at creation."""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import check_outputs, close, force_weights, fw_of, random_state

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-10, 2: 1e-4, 3: 1e-4}


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


def clouds(nx, ny, seed, geometry=0):
    c = wl.lognormal_cloud(nx, ny, seed=seed, v_edge_kms=60.0, Z=0.1, p_d=1e-7)
    c.temp = wl.two_phase_temperature(nx, ny, seed + 1, T_cold=80.0, T_hot=2e4)
    c.geometry = geometry
    if geometry == 1:
        c.bc = (0, 1, 0, 1)
    T1 = wl.two_phase_temperature(nx, ny, seed + 2, T_cold=300.0, T_hot=8e3)
    return c, T1


@pytest.mark.parametrize("geometry", [0, 1])
@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_substeps_after_new_temperatures_match_oracle(L, edges, precision, geometry):
    c, T1 = clouds(45, 38, seed=121, geometry=geometry)
    st = random_state(194, 38, 45, 124)
    ctx = L.from_cloud(c, precision=precision, edges=edges)
    ctx.set_state(*st)
    ctx.substeps(2)
    ctx.set_temperature(T1)
    ctx.substeps(3)
    got = ctx.get_state() + ctx.force()
    ctx.destroy()
    O0 = oracle.Oracle(edges=edges, **c.kwargs())
    J, Hx, Hy = st
    for _ in range(2):
        J, Hx, Hy, _, _, _ = O0.substep(J, Hx, Hy)
    c.temp = T1
    O1 = oracle.Oracle(edges=edges, **c.kwargs())
    (J, Hx, Hy, fx, fy), _ = O1.run(3, (J, Hx, Hy))
    check_outputs(got, (J, Hx, Hy, fx, fy), TOL[precision], 5, st, force_weights(O1, c.dx))


@pytest.mark.parametrize("precision", [1, 3])
def test_device_tables_agree_with_host_tables(L, edges, precision):
    c, T1 = clouds(40, 24, seed=131)
    st = random_state(194, 24, 40, 134)
    dev = L.from_cloud(c, precision=precision, edges=edges)
    dev.set_temperature(T1)
    c.temp = T1
    host = L.from_cloud(c, precision=precision, edges=edges)
    for x in (dev, host):
        x.set_state(*st)
        x.substeps(3)
    bar = 1e-12 if precision == 1 else 1e-5
    check_outputs(dev.get_state() + dev.force(), host.get_state() + host.force(), bar, 3, st, fw_of(c, edges))
    dev.destroy()
    host.destroy()


def test_gray_group_with_new_temperatures(L, edges):
    c = wl.uniform_gray(40, 28)
    c.temp = wl.two_phase_temperature(40, 28, seed=141)
    T1 = wl.two_phase_temperature(40, 28, seed=142, T_cold=500.0, T_hot=3e4)
    ctx = L.from_cloud(c, precision=1, edges=edges)
    ctx.substeps(5)
    ctx.set_temperature(T1)
    ctx.substeps(5)
    got = ctx.get_state() + ctx.force()
    ctx.destroy()
    O0 = oracle.Oracle(edges=edges, **c.kwargs())
    (J, Hx, Hy, _, _), _ = O0.run(5)
    c.temp = T1
    (J, Hx, Hy, fx, fy), _ = oracle.Oracle(edges=edges, **c.kwargs()).run(5, (J, Hx, Hy))
    for a, b, n in zip(got, (J, Hx, Hy, fx, fy), ("J", "Hx", "Hy", "fx", "fy")):
        close(a, b, 1e-10, n)


def test_set_temperature_rejects(L, edges):
    c, T1 = clouds(16, 16, seed=151)
    ctx = L.from_cloud(c, precision=3, edges=edges)
    ctx.substeps(2)
    before = ctx.get_state()
    for bad in (0.0, -3.0, float("nan"), float("inf")):
        T = T1.copy()
        T[5, 7] = bad
        with pytest.raises(L.Lym1Error) as e:
            ctx.set_temperature(T)
        assert e.value.status == L.EINVAL
    for u, w in zip(ctx.get_state(), before):
        np.testing.assert_array_equal(u, w)
    ctx.destroy()
    plain = L.from_cloud(wl.lognormal_cloud(16, 16, seed=152), precision=3, edges=edges)
    with pytest.raises(L.Lym1Error) as e:
        plain.set_temperature(T1)
    assert e.value.status == L.EINVAL
    plain.destroy()

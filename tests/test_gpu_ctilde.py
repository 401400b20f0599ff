"""Dynamic reduced speed of light on the GPU (Sec. 2.1: the dynamic-RSL rule,
its f_abs factor, the c_min floor, the c cap and the -25 % / x4 rate limits)
against the oracle, and the substeps that follow a change of c_tilde: the
RT time step and every c_tilde-dependent coefficient of the graph-replayed
and batched paths must move with it (bit-exact in LYM1_FP64_DET, the
test_gpu_parity bars otherwise).  The c_tilde values agree to 1e-14: the
kernel and the oracle differ only in the rounding of the cube root."""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import TOL, check_outputs, close, force_weights, random_state

pytestmark = pytest.mark.gpu

KM = 1.0e5
C = 2.99792458e10


@pytest.fixture(scope="module")
def L():
    import paper_2606_02711_gb300.lym1 as L
    L.lib()
    return L


@pytest.fixture(scope="module")
def edges():
    return oracle.freq_grid()


@pytest.mark.parametrize("case", ["cart", "cyl", "temperature", "cs_host", "cs_device"])
def test_dynamic_ctilde_matches_oracle(L, edges, case):
    nx, ny = 45, 38
    c = wl.lognormal_cloud(nx, ny, seed=91, v_edge_kms=20.0, Z=0.3, p_d=1e-6)
    cs = cs_arg = None
    if case == "cyl":
        c.geometry, c.bc = 1, (0, 1, 0, 1)
    if case == "temperature":
        c.temp = wl.two_phase_temperature(nx, ny, seed=92, T_cold=80.0, T_hot=2e4)
    if case.startswith("cs"):
        cs = np.random.default_rng(93).uniform(1.0, 30.0, (ny, nx)) * KM
        cs_arg = cs
        if case == "cs_device":
            torch = pytest.importorskip("torch")
            cs_arg = torch.tensor(cs, dtype=torch.float64, device="cuda")
    ctx = L.from_cloud(c, precision="mixed_fast", edges=edges)
    O = oracle.Oracle(edges=edges, **c.kwargs())
    seq = []
    # from c down through the -25 % steps to the rule's own value
    for _ in range(40):
        a = ctx.dynamic_ctilde(cs=cs_arg)
        b = O.dynamic_ctilde(cs=cs)
        assert a == pytest.approx(b, rel=1e-14, abs=0)
        assert ctx.dt_cfl == pytest.approx(O.dt_cfl, rel=1e-14, abs=0)
        seq.append(a)
    ctx.destroy()
    assert seq[0] == 0.75 * C
    # -25 % steps until the rule's value is within reach, then that value
    k = next(i for i in range(1, len(seq)) if seq[i] != 0.75 * seq[i - 1])
    assert all(v == seq[k] for v in seq[k:])
    assert 0.75 * seq[k - 1] < seq[k] < seq[k - 1]
    # the optically thick cells set it: well above eps_RSL x the fastest speed
    umax = float(np.hypot(c.ux, c.uy).max())
    assert seq[-1] > 8.0 * max(umax, 30.0 * KM)


@pytest.mark.parametrize("precision", [0, 1, 3])
def test_substeps_follow_new_ctilde(L, edges, precision):
    c = wl.lognormal_cloud(37, 29, seed=94, v_edge_kms=40.0)
    st = random_state(194, 29, 37, 95)
    ctx = L.from_cloud(c, precision=precision, edges=edges)
    ctx.set_state(*st)
    O = oracle.Oracle(edges=edges, **c.kwargs())
    J, Hx, Hy = st
    # graph-replayed substeps at c, then a new c_tilde, then more substeps
    ctx.substeps(2)
    for _ in range(2):
        J, Hx, Hy, fx, fy, _ = O.substep(J, Hx, Hy)
    done = 2
    for set_ct in ("dynamic", 2.0e9):
        if set_ct == "dynamic":
            ct = ctx.dynamic_ctilde(ct_min=0.0)
            O.set_ctilde(ct)
            assert ct == 0.75 * C
        else:
            ctx.set_ctilde(set_ct)
            O.set_ctilde(set_ct)
        assert ctx.dt_cfl == O.dt_cfl
        ctx.substeps(3)
        done += 3
        for _ in range(3):
            J, Hx, Hy, fx, fy, _ = O.substep(J, Hx, Hy)
        got = ctx.get_state() + ctx.force()
        check_outputs(got, (J, Hx, Hy, fx, fy), TOL[precision], done, st, force_weights(O, c.dx))
    ctx.destroy()


def test_batch_picks_up_new_ctilde(L, edges):
    clouds = [wl.lognormal_cloud(40, 24, seed=96), wl.lognormal_cloud(17, 33, seed=97)]
    solo = []
    for i, c in enumerate(clouds):
        x = L.from_cloud(c, precision="mixed_fast", edges=edges)
        x.substeps(2)
        if i == 0:
            x.set_ctilde(3.0e9)
        x.substeps(3)
        solo.append(x.get_state())
        x.destroy()
    ctxs = [L.from_cloud(c, precision="mixed_fast", edges=edges) for c in clouds]
    b = L.Batch(ctxs)
    b.substeps(2)
    ctxs[0].set_ctilde(3.0e9)
    b.substeps(3)
    b.destroy()
    for x, s in zip(ctxs, solo):
        for u, w in zip(x.get_state(), s):
            np.testing.assert_array_equal(u, w)
        x.destroy()


def test_invalid_arguments_leave_ctilde_unchanged(L, edges):
    c = wl.lognormal_cloud(16, 16, seed=98)
    ctx = L.from_cloud(c, precision="mixed_fast", edges=edges)
    dt = ctx.dt_cfl
    for bad in (0.0, -1.0, 1.01 * C, float("nan")):
        with pytest.raises(L.Lym1Error) as e:
            ctx.set_ctilde(bad)
        assert e.value.status == L.EINVAL
    for kw in ({"eps_rsl": 0.0}, {"eps_rsl": float("inf")}, {"ct_min": -1.0},
               {"ct_min": 2 * C}):
        with pytest.raises(L.Lym1Error) as e:
            ctx.dynamic_ctilde(**kw)
        assert e.value.status == L.EINVAL
    assert ctx.info()["dt_cfl"] == dt
    ctx.destroy()

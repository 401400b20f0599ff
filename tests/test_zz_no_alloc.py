"""lym1_energy_noalloc: the allocation-free energy of a caller-owned state.

It serves callers that cannot allocate device memory when they need the
number (memory owned by another runtime's allocator, real-time loops, work
recorded into a CUDA graph).  This file sorts last so that a run stopping at
its first failure has already run every other test.  It checks the call
against the energy that lym1_diagnostics reports for the same state (the
existing entry point), on two calls in a row, and its size limits.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _state(seed, nb, ny, nx):
    g = np.random.default_rng(seed)
    J = 1e-12 * np.exp(g.normal(0.0, 1.0, (nb, ny, nx)))
    f = g.uniform(0.0, 0.9, (nb, ny, nx))
    return J, 0.6 * f * J, -0.7 * f * J


def test_energy_noalloc_matches_diagnostics_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L

    c = wl.lognormal_cloud(45, 38, seed=3)
    ctx = L.from_cloud(c, precision=L.FP64_DET)
    dnu = ctx.tables()["dnu"]
    values = []
    for seed in (11, 12):  # two calls in a row, different states
        st = _state(seed, ctx.nb, c.ny, c.nx)
        ctx.set_state(*st)
        ref = ctx.diagnostics()["e_tot"]
        Jd = torch.from_numpy(st[0]).to("cuda")
        got = L.energy_noalloc(Jd, dnu, c.dx)
        assert got == pytest.approx(ref, rel=1e-12)
        values.append(got)
    assert values[0] != values[1]
    ctx.destroy()


def test_energy_noalloc_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L

    lib = L.lib()
    J = torch.zeros(8, dtype=torch.float64, device="cuda")
    Jp = C.cast(C.c_void_p(J.data_ptr()), C.POINTER(C.c_double))
    out = np.zeros(1)
    op = out.ctypes.data_as(C.POINTER(C.c_double))
    dnu = np.ones(2000)
    dp = dnu.ctypes.data_as(C.POINTER(C.c_double))
    # the size checks come before any device access
    assert lib.lym1_energy_noalloc(Jp, dp, 2000, 1, 1.0, op, None) == L.ERANGE
    assert lib.lym1_energy_noalloc(Jp, dp, 1, (1 << 24) + 1, 1.0, op, None) == L.ERANGE
    assert lib.lym1_energy_noalloc(Jp, dp, 0, 8, 1.0, op, None) == L.EINVAL
    assert lib.lym1_energy_noalloc(Jp, dp, 1, 8, 1.0, op, None) == L.OK
    assert out[0] == 0.0

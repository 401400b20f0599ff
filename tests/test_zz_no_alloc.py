"""lym1_energy_noalloc: the allocation-free energy of a caller-owned state.

The call serves callers that cannot allocate device memory when they need the
number: a host code whose HBM is already reserved by another runtime's
allocator, or a real-time loop that forbids allocation.  This file sorts last
so that a run stopping at its first failure has already run every other test.
It checks the call against the energy that lym1_diagnostics reports for the
same state (the existing entry point), on two calls in a row, bit for bit: the
two use the same partition, order and rounding for an FP64 Cartesian context.
It also checks that repeated calls leave the device's free memory unchanged,
that host arrays are refused before any launch, and the size limits.
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


# 45 x 38 = 14 blocks of partial sums; 256 x 256 = 512 blocks, so the second
# stage's strided loop (256 threads) takes two partials per thread
@pytest.mark.parametrize("nx,ny", [(45, 38), (256, 256)])
def test_energy_noalloc_matches_diagnostics_on_two_calls(nx, ny):
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L

    c = wl.lognormal_cloud(nx, ny, seed=3)
    ctx = L.from_cloud(c, precision=L.FP64_DET)
    dnu = ctx.tables()["dnu"]
    values = []
    for seed in (11, 12):  # two calls in a row, different states
        st = _state(seed, ctx.nb, c.ny, c.nx)
        ctx.set_state(*st)
        ref = ctx.diagnostics()["e_tot"]
        Jd = torch.from_numpy(st[0]).to("cuda")
        got = L.energy_noalloc(Jd, dnu, c.dx)
        assert got == ref, (got, ref)
        values.append(got)
    assert values[0] != values[1]
    ctx.destroy()


def test_energy_noalloc_allocates_nothing():
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L

    g = np.random.default_rng(5)
    dnu = g.uniform(1e9, 2e9, 194)
    shapes = [(194, 64, 64), (194, 300, 200), (7, 1024, 1024), (1, 1, 1)]
    Js = [torch.from_numpy(1e-12 * g.random(s)).to("cuda") for s in shapes]
    torch.cuda.synchronize()
    L.energy_noalloc(Js[0], dnu[:194], 1e17)  # first call: looks up the scratch address
    free0 = torch.cuda.mem_get_info()[0]
    out = []
    for J, s in zip(Js, shapes):
        for _ in range(3):
            out.append(L.energy_noalloc(J, dnu[:s[0]], 1e17))
    assert torch.cuda.mem_get_info()[0] == free0
    # the value does not depend on what earlier calls left in the shared array
    assert out[0] == out[1] == out[2] and out[3] == out[4] == out[5]


def test_energy_noalloc_refuses_host_memory():
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L

    lib = L.lib()
    out = np.full(1, -1.0)
    op = out.ctypes.data_as(C.POINTER(C.c_double))
    dnu = np.ones(2)
    dp = dnu.ctypes.data_as(C.POINTER(C.c_double))
    host = np.ones(16)
    pinned = torch.ones(16, dtype=torch.float64).pin_memory()
    for buf in (host.ctypes.data_as(C.POINTER(C.c_double)),
                C.cast(C.c_void_p(pinned.data_ptr()), C.POINTER(C.c_double))):
        assert lib.lym1_energy_noalloc(buf, dp, 2, 8, 1.0, op, None) == L.EINVAL
    assert out[0] == -1.0
    with pytest.raises(ValueError):
        L.energy_noalloc(torch.ones(16, dtype=torch.float64), dnu, 1.0)
    with pytest.raises(ValueError):  # 15 values are not 2 x nc
        L.energy_noalloc(torch.ones(15, dtype=torch.float64, device="cuda"), dnu, 1.0)
    # the context stays usable: a valid call right after
    Jd = torch.ones(16, dtype=torch.float64, device="cuda")
    assert L.energy_noalloc(Jd, dnu, 1.0) > 0.0


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

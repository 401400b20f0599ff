"""The FP64 helpers of the LYM1_MIXED kernels against IEEE-754 arithmetic.

GB300 runs FP64 arithmetic and FP32 <-> FP64 conversions on a pipe of about
1/70 of the FP32 rate, so the mixed kernels widen and narrow on the integer
pipe and refine the hardware reciprocal approximation by Newton-Raphson.
Widening must be exact and narrowing correctly rounded (to nearest, ties to
even) wherever the result is a binary32 normal number or infinity; both flush
subnormals to zero.  The reciprocal must lie within one ulp of 1/x; the one-step reciprocal
(whose results are rounded to FP32) within 2^-38 of it, and the FP32-seeded one
of the mixed source step and elimination within 2^-40 over the normal range.  numpy's
conversions and division are the IEEE reference.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FLT_MIN = np.float32(np.finfo(np.float32).tiny)


def _run(xf, xd):
    torch = pytest.importorskip("torch")
    import paper_2606_02711_gb300.lym1 as L
    n = xf.size
    assert xd.size == n
    a = torch.from_numpy(xf).cuda()
    b = torch.from_numpy(xd).cuda()
    wide = torch.empty(n, dtype=torch.float64, device="cuda")
    narrow = torch.empty(n, dtype=torch.float32, device="cuda")
    rcp = torch.empty(n, dtype=torch.float64, device="cuda")
    rcp1 = torch.empty(n, dtype=torch.float64, device="cuda")
    rcpf = torch.empty(n, dtype=torch.float64, device="cuda")
    st = L.lib().lym1_debug_fp64_helpers(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), n,
                                         C.c_void_p(wide.data_ptr()), C.c_void_p(narrow.data_ptr()),
                                         C.c_void_p(rcp.data_ptr()), C.c_void_p(rcp1.data_ptr()),
                                         C.c_void_p(rcpf.data_ptr()))
    assert st == 0
    _run.rcp1 = rcp1.cpu().numpy()
    _run.rcpf = rcpf.cpu().numpy()
    return wide.cpu().numpy(), narrow.cpu().numpy(), rcp.cpu().numpy()


def _bits32(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def _bits64(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def test_widening_is_exact_and_flushes_subnormals():
    g = np.random.default_rng(1)
    n = 1 << 20
    u = g.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    xf = u.view(np.float32).copy()
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, FLT_MIN, -FLT_MIN,
                         np.finfo(np.float32).max, 1e-45, -3e-39, 1.0, -2.5], dtype=np.float32)
    xf[:specials.size] = specials
    wide, _, _ = _run(xf, np.ones(n))
    ref = xf.astype(np.float64)
    nan = np.isnan(xf)
    sub = (np.abs(xf) < FLT_MIN) & (xf != 0)
    ok = ~nan & ~sub
    assert np.array_equal(_bits64(wide[ok]), _bits64(ref[ok]))
    assert np.all(np.isnan(wide[nan]))
    assert np.all(wide[sub] == 0.0)
    assert np.array_equal(np.signbit(wide[sub]), np.signbit(xf[sub]))


def test_narrowing_rounds_to_nearest_even():
    g = np.random.default_rng(2)
    n = 1 << 20
    # random doubles over the binary32 range and somewhat beyond
    e = g.uniform(-140.0, 130.0, n)
    xd = np.where(g.random(n) < 0.5, -1.0, 1.0) * 2.0 ** e * g.uniform(1.0, 2.0, n)
    # exact ties between two binary32 neighbours, with even and odd lower neighbours
    m = g.integers(1 << 23, 1 << 24, 4096)
    k = g.integers(-100, 100, 4096)
    ties = (m.astype(np.float64) + 0.5) * 2.0 ** (k - 23)
    xd[:4096] = ties
    # just below and above a tie, and at the top of the range
    xd[4096:8192] = np.nextafter(ties, 0.0)
    xd[8192:12288] = np.nextafter(ties, np.inf)
    fmax = float(np.finfo(np.float32).max)
    xd[12288:12300] = [fmax, fmax * (1 + 2 ** -25), fmax * (1 + 2 ** -23), 1e39, -1e300, np.inf,
                       -np.inf, np.nan, 0.0, -0.0, 1e-300, float(FLT_MIN)]
    _, narrow, _ = _run(np.ones(n, dtype=np.float32), xd)
    with np.errstate(over="ignore"):
        ref = xd.astype(np.float32)
    nan = np.isnan(xd)
    tiny = np.abs(ref) < FLT_MIN
    ok = ~nan & ~tiny
    assert np.array_equal(_bits32(narrow[ok]), _bits32(ref[ok]))
    assert np.all(np.isnan(narrow[nan]))
    assert np.all(narrow[tiny] == 0.0)
    assert np.array_equal(np.signbit(narrow[tiny]), np.signbit(xd[tiny]))


def test_reciprocal_within_one_ulp():
    g = np.random.default_rng(3)
    n = 1 << 20
    xd = 10.0 ** g.uniform(-300.0, 300.0, n) * g.uniform(1.0, 10.0, n)
    xd[:6] = [1.0, 2.0, 3.0, 1.0 + 2 ** -52, 1e300, 7.0]
    _, _, rcp = _run(np.ones(n, dtype=np.float32), xd)
    ref = 1.0 / xd
    ulp = np.abs(_bits64(rcp).astype(np.int64) - _bits64(ref).astype(np.int64))
    assert ulp.max() <= 1
    assert np.mean(ulp == 0) > 0.9


def test_one_step_reciprocal_within_2_pow_minus_38():
    # the one Newton step squares the approximation's relative error: the
    # bound the mixed source and elimination steps rely on, far below the FP32
    # rounding (2^-24) their results then take
    g = np.random.default_rng(4)
    n = 1 << 20
    xd = 10.0 ** g.uniform(-300.0, 300.0, n) * g.uniform(1.0, 10.0, n)
    xd[:6] = [1.0, 2.0, 3.0, 1.0 + 2 ** -52, 1e300, 7.0]
    _run(np.ones(n, dtype=np.float32), xd)
    rel = np.abs(_run.rcp1 * xd - 1.0)
    assert rel.max() <= 2.0 ** -38, f"max relative error 2^{np.log2(rel.max()):.1f}"


def test_fp32_seeded_reciprocal_within_2_pow_minus_40():
    # the mixed source step's denominators 1 + c dt kappa, 1 + c dt alpha_F and
    # the elimination's pivots: the seed is the FP32 SFU reciprocal of the
    # significand (exponent handled apart, so any normal x below 2^1020), and
    # one FP64 Newton step squares its error
    g = np.random.default_rng(5)
    n = 1 << 20
    xd = 10.0 ** g.uniform(-300.0, 300.0, n) * g.uniform(1.0, 10.0, n)
    xd[:12] = [1.0, 1.0 + 2 ** -52, 2.0 - 2 ** -52, 2.0, 3.0, 1e30, 7.0, 2.0 ** 1019,
               2.0 ** -1021, 1.5 * 2.0 ** -1000, np.nextafter(1.0, 0.0), 1e-5]
    _run(np.ones(n, dtype=np.float32), xd)
    rel = np.abs(_run.rcpf * xd - 1.0)
    assert rel.max() <= 2.0 ** -40, f"max relative error 2^{np.log2(rel.max()):.1f}"

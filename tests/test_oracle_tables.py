"""Pins for the oracle's setup step A0 (frequency grid, line constants, bin-averaged
Voigt profile, emission fractions) and for its own exp/expm1/Dawson routines.

Each check compares against something fixed outside the oracle: numbers the
paper prints, scipy's special functions and quadrature, closed-form limits.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle

SQRTPI = math.sqrt(math.pi)


def test_paper_grid_has_194_bins(paper_edges):
    # Sec. 2.1: q = 1.1, T_min = 30 K "yields N_nu = 194 frequency bins"
    assert paper_edges.size - 1 == 194


def test_grid_shape(paper_edges):
    e = paper_edges
    w = np.diff(e)
    dnuD30 = oracle.line_constants(30.0)["dnu_D"]
    M = w.size // 2
    # symmetric about line centre, centre edge exactly 0
    assert e[M] == 0.0
    np.testing.assert_array_equal(e[::-1], -e)
    # the two central bins have width dnu_D(T_min), widths grow by q = 1.1 outwards
    assert w[M] == pytest.approx(dnuD30, rel=1e-15)
    ratios = w[M + 1:-1] / w[M:-2]
    np.testing.assert_allclose(ratios, 1.1, rtol=1e-12)
    # |dnu| <= 1e5 dnu_D(T_min), the binding limit (< nu_LyC - nu_Lya)
    assert e[-1] == pytest.approx(1e5 * dnuD30, rel=1e-15)
    assert w[-1] < 1.1 * w[-2]


def test_finer_grid_count():
    # Sec. 2.1 Test 2 quotes 594 bins for q = 1.03; the stated truncation rule
    # gives 542 (reading recorded in the design notes).  The rule is pinned here.
    e = oracle.freq_grid(30.0, 1.03)
    assert e.size - 1 == 542


@pytest.mark.parametrize("T", [1e2, 1e3, 1e4, 3e4])
def test_line_constants_match_printed_scalings(T):
    # Sec. 2.1: a_v ~ 4.7e-4 T4^-1/2, tau0 ~ 5.9e-14 T4^-1/2 N_HI
    lc = oracle.line_constants(T)
    T4 = T / 1e4
    assert lc["a_v"] == pytest.approx(4.7e-4 / math.sqrt(T4), rel=0.01)
    assert lc["sigma0"] == pytest.approx(5.9e-14 / math.sqrt(T4), rel=0.01)
    # Doppler width from the thermal speed sqrt(2 kT / m_H): 12.85 km/s at 1e4 K
    assert lc["dnu_D"] / 2.466e15 * 2.99792458e5 == pytest.approx(12.85 * math.sqrt(T4), rel=2e-3)


def test_dawson_against_scipy():
    xs = np.concatenate([np.linspace(-12, 12, 2401), [1e-8, 0.1999999, 0.2, 9.999999, 10.0,
                                                       50.0, 1e3, 5e3, 1e5]])
    for x in xs:
        ref = sp.dawsn(x)
        got = oracle.dawson(x)
        assert abs(got - ref) <= 4e-15 * max(abs(ref), 1e-300) + 1e-300, x


def _ulps(a, b):
    if a == b:
        return 0
    ia = np.frombuffer(np.float64(a).tobytes(), np.int64)[0]
    ib = np.frombuffer(np.float64(b).tobytes(), np.int64)[0]
    return abs(int(ia) - int(ib))


def test_own_exp_expm1_against_libm():
    g = np.random.default_rng(5)
    xs = np.concatenate([-np.logspace(-12, math.log10(744), 4000), np.linspace(-1, 1, 2001),
                         g.uniform(-745, 5, 4000), [0.0, -0.0, -0.3465735902799726,
                                                    0.3465735902799726, -708.5, -744.9]])
    worst_e = worst_m = 0
    for x in xs:
        worst_e = max(worst_e, _ulps(oracle.exp(x), math.exp(x)))
        m = math.expm1(x)
        if abs(m) > 1e-300:
            worst_m = max(worst_m, _ulps(oracle.expm1(x), m))
    # Cody-Waite + degree-13 Taylor: within 2 ulp of glibc everywhere (subnormal
    # results included, where one ulp is the absolute spacing)
    assert worst_e <= 2
    assert worst_m <= 2


def _voigt_expansion(x, a):
    # derivative of I(x,a) in App. A: the second-order expansion of H in a
    F = sp.dawsn(x)
    return (math.exp(-x * x) - (2 * a / SQRTPI) * (1 - 2 * x * F)
            + a * a * (1 - 2 * x * x) * math.exp(-x * x))


def test_bin_average_matches_quadrature(paper_edges):
    T = 1e4
    t = oracle.bin_tables(paper_edges, T)
    lc = oracle.line_constants(T)
    dnuD, a = lc["dnu_D"], lc["a_v"]
    xe = paper_edges / dnuD
    # quadrature of 1 - 2xF(x) loses digits beyond |x| ~ 100, where the wing
    # limit in test_profile_limits_and_normalisation takes over
    ks = [k for k in range(xe.size - 1) if max(abs(xe[k]), abs(xe[k + 1])) < 100.0]
    assert len(ks) > 60
    for k in ks:
        xa, xb = xe[k], xe[k + 1]
        pts = [0.0] if xa < 0 < xb else None
        val, _ = si.quad(_voigt_expansion, xa, xb, args=(a,), epsabs=0, epsrel=1e-13,
                         limit=400, points=pts)
        ref = val / (xb - xa)
        assert t["Havg"][k] == pytest.approx(ref, rel=1e-10, abs=0), k


def test_bin_average_matches_exact_voigt(paper_edges):
    # H(a,x) = sqrt(pi) * Voigt(x; sigma=1/sqrt(2), gamma=a); the expansion is
    # accurate to O(a^3) in the core and to O(a x^-4) relative in the wings.
    T = 1e4
    t = oracle.bin_tables(paper_edges, T)
    lc = oracle.line_constants(T)
    dnuD, a = lc["dnu_D"], lc["a_v"]
    xe = paper_edges / dnuD
    for k in range(60, 134):
        xa, xb = xe[k], xe[k + 1]
        f = lambda x: SQRTPI * sp.voigt_profile(x, 1 / math.sqrt(2), a)
        pts = [0.0] if xa < 0 < xb else None
        val, _ = si.quad(f, xa, xb, epsabs=0, epsrel=1e-12, limit=400, points=pts)
        assert t["Havg"][k] == pytest.approx(val / (xb - xa), rel=2e-6), k


def test_profile_limits_and_normalisation(paper_edges):
    T = 1e4
    t = oracle.bin_tables(paper_edges, T)
    lc = oracle.line_constants(T)
    dnuD, a = lc["dnu_D"], lc["a_v"]
    xe = paper_edges / dnuD
    dx = np.diff(xe)
    # telescoping: sum dx_k <H>_k = I(x_N) - I(x_0) -> sqrt(pi) - 4a F(x_max)/sqrt(pi)
    S = float(np.sum(dx * t["Havg"]))
    ref = SQRTPI - 2 * (2 * a / SQRTPI) * sp.dawsn(xe[-1])
    assert S == pytest.approx(ref, rel=1e-13)
    # line centre: bin width 0.055 Doppler widths, H(0) = 1 - 2a/sqrt(pi) + a^2
    M = t["Havg"].size // 2
    xb = xe[M + 1]
    center = (SQRTPI / 2 * math.erf(xb) / xb)  # Gaussian core averaged over the bin
    assert t["Havg"][M] == pytest.approx(center - 2 * a / SQRTPI, rel=1e-5)
    # far wings: bin average of a/(sqrt(pi) x^2) = a / (sqrt(pi) xa xb)
    for k in (0, 5, 20):
        xa_, xb_ = abs(xe[k + 1]), abs(xe[k])
        assert t["Havg"][k] == pytest.approx(a / (SQRTPI * xa_ * xb_), rel=2e-6)
    # emission fractions sum to one and are symmetric; eta ~ 1/sqrt(2) (Sec. 4, Test 1)
    assert t["w"].sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(t["w"], t["w"][::-1], rtol=1e-13)
    np.testing.assert_allclose(t["Havg"], t["Havg"][::-1], rtol=1e-13)
    assert t["eta"] == pytest.approx(1 / math.sqrt(2), rel=0.01)

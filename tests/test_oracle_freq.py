"""Pins for the oracle's frequency step A6 (App. A): exponential-scheme leakage
coefficients, the BDF1 tridiagonal solve, conservation, limits and equilibria.

References used here are independent of the oracle's code: the App. A
coefficient formulas evaluated directly with numpy at moderate Peclet numbers,
dense and exact-rational linear solves, scipy's banded solver for the
central-difference limit, and the zero-flux equilibrium of the scheme.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle

C = 2.99792458e10


def _coeffs(edges, T, alpha, recoil, DdU):
    """Per-bin K_k, C_k, P_k, half widths dlt_k, widths dnu_k (App. A)."""
    lc = oracle.line_constants(T)
    t = oracle.bin_tables(edges, T)
    dnu, nubar, Hv = t["dnu"], t["nubar"], t["Havg"]
    hkT = 6.62607015e-27 / (1.380649e-16 * T)
    R = (hkT - 2.0 / nubar) if recoil else np.zeros_like(nubar)
    K = 0.5 * lc["dnu_D"] ** 2 * alpha * Hv
    Cc = K * R + nubar / C * np.broadcast_to(DdU, K.shape)
    dlt = 0.5 * dnu
    return K, Cc, Cc * dlt / K, dlt, dnu


def _paper_matrix(edges, T, alpha, recoil, DdU, cdt):
    """The App. A system (J - Jin)/(ct dt) = F+ J_{k+1} - F J_k + F- J_{k-1}
    written straight from the leakage-coefficient formulas."""
    K, Cc, P, dlt, dnu = _coeffs(edges, T, alpha, recoil, DdU)
    N = K.size
    phiL = lambda x: -np.expm1(-x)
    phiR = lambda x: -np.expm1(x)
    chiL = lambda x: phiL(x) / x if x != 0 else 1.0
    chiR = lambda x: phiR(x) / x if x != 0 else -1.0
    den = np.array([chiL(P[k]) * dlt[k] / K[k] - chiR(P[k + 1]) * dlt[k + 1] / K[k + 1]
                    for k in range(N - 1)])
    Fp, Fm, F = np.zeros(N), np.zeros(N), np.zeros(N)
    for k in range(N):
        if k + 1 < N:
            Fp[k] = (1 - phiR(P[k + 1])) / den[k] / dnu[k]
            F[k] += (1 - phiL(P[k])) / den[k] / dnu[k]
        if k > 0:
            Fm[k] = (1 - phiL(P[k - 1])) / den[k - 1] / dnu[k]
            F[k] += (1 - phiR(P[k])) / den[k - 1] / dnu[k]
    M = np.diag(1.0 / cdt + F) - np.diag(Fp[:-1], 1) - np.diag(Fm[1:], -1)
    return M, P


def _toy_grid(N=30, width_dop=0.5, T=1e4):
    dnuD = oracle.line_constants(T)["dnu_D"]
    return (np.arange(N + 1) - N / 2) * width_dop * dnuD


def _ddu_for_peclet(edges, T, alpha, Ptarget):
    K, Cc, P, dlt, dnu = _coeffs(edges, T, alpha, False, 0.0)
    nubar = oracle.bin_tables(edges, T)["nubar"]
    return Ptarget * K / dlt / (nubar / C)


def test_leakage_matches_paper_formulas_at_moderate_peclet():
    T, alpha = 1e4, 1e-9
    e = _toy_grid()
    g = np.random.default_rng(3)
    for trial in range(6):
        Pt = g.uniform(-30, 30, e.size - 1) if trial else np.zeros(e.size - 1)
        ddu = _ddu_for_peclet(e, T, alpha, Pt)
        A, B = oracle.leakage(e, T, alpha, True, ddu)
        K, Cc, P, dlt, dnu = _coeffs(e, T, alpha, True, ddu)
        for k in range(e.size - 2):
            chiL = -math.expm1(-P[k]) / P[k] if P[k] else 1.0
            chiR = -math.expm1(P[k + 1]) / P[k + 1] if P[k + 1] else -1.0
            den = chiL * dlt[k] / K[k] - chiR * dlt[k + 1] / K[k + 1]
            assert A[k] == pytest.approx(math.exp(-P[k]) / den, rel=2e-13)
            assert B[k] == pytest.approx(math.exp(P[k + 1]) / den, rel=2e-13)


def test_leakage_limits_central_and_upwind():
    T, alpha = 1e4, 1e-9
    e = _toy_grid()
    K, Cc, P, dlt, dnu = _coeffs(e, T, alpha, False, 0.0)
    # P -> 0: central difference, A = B = 1 / (dlt_k/K_k + dlt_{k+1}/K_{k+1})
    A, B = oracle.leakage(e, T, alpha, False, 0.0)
    G = 1.0 / (dlt[:-1] / K[:-1] + dlt[1:] / K[1:])
    np.testing.assert_allclose(A, G, rtol=1e-15)
    np.testing.assert_allclose(B, G, rtol=1e-15)
    # |P| >> 1 (no overflow even at P ~ 1e5): upwinding, flux = C_donor J_donor
    for Pt in (800.0, 1e5):
        ddu = _ddu_for_peclet(e, T, alpha, np.full(e.size - 1, Pt))
        A, B = oracle.leakage(e, T, alpha, False, ddu)
        K, Cc, P, dlt, dnu = _coeffs(e, T, alpha, False, ddu)
        assert np.all(np.isfinite(A)) and np.all(np.isfinite(B))
        np.testing.assert_allclose(B, Cc[1:], rtol=2.0 / Pt)
        assert np.all(A <= 1e-300 + 1e-12 * B)
        ddu = _ddu_for_peclet(e, T, alpha, np.full(e.size - 1, -Pt))
        A, B = oracle.leakage(e, T, alpha, False, ddu)
        K, Cc, P, dlt, dnu = _coeffs(e, T, alpha, False, ddu)
        np.testing.assert_allclose(A, -Cc[:-1], rtol=2.0 / Pt)
        assert np.all(B <= 1e-300 + 1e-12 * A)


@pytest.mark.parametrize("cdt", [1e8, 1e11])
def test_solve_matches_dense_paper_system(cdt):
    T, alpha = 1e4, 1e-9
    e = _toy_grid()
    g = np.random.default_rng(4)
    ddu = _ddu_for_peclet(e, T, alpha, g.uniform(-20, 20, e.size - 1))
    Jin = g.uniform(0.5, 2.0, e.size - 1)
    M, P = _paper_matrix(e, T, alpha, True, ddu, cdt)
    ref = np.linalg.solve(M, Jin / cdt)
    got = oracle.freq_solve(e, T, alpha, True, ddu, cdt, Jin)
    np.testing.assert_allclose(got, ref, rtol=1e-9 if cdt > 1e9 else 1e-12)


def _exact_solve(A, B, s, rhs):
    """Exact rational solve of the conservative tridiagonal system."""
    N = len(s)
    M = [[Fraction(0)] * N for _ in range(N)]
    for k in range(N):
        M[k][k] = s[k] + (A[k] if k + 1 < N else 0) + (B[k - 1] if k > 0 else 0)
        if k + 1 < N:
            M[k][k + 1] = -B[k]
        if k > 0:
            M[k][k - 1] = -A[k - 1]
    b = list(rhs)
    for i in range(N):
        piv = M[i][i]
        for r in range(i + 1, N):
            if M[r][i] != 0:
                fac = M[r][i] / piv
                for c in range(i, N):
                    M[r][c] -= fac * M[i][c]
                b[r] -= fac * b[i]
    x = [Fraction(0)] * N
    for i in reversed(range(N)):
        acc = b[i] - sum(M[i][c] * x[c] for c in range(i + 1, N))
        x[i] = acc / M[i][i]
    return x


@pytest.mark.parametrize("cdt", [1e14, 1e18, 1e22])
def test_stiff_solve_against_exact_rational(cdt):
    # the stiff regime (ct dt F ~ 1e7..1e15): the subtraction-free elimination
    # keeps full relative accuracy; checked against exact rational arithmetic
    T, alpha = 1e4, 1e-7
    e = _toy_grid(N=14, width_dop=0.8)
    g = np.random.default_rng(9)
    ddu = _ddu_for_peclet(e, T, alpha, g.uniform(-3, 3, e.size - 1))
    Jin = g.uniform(0.1, 3.0, e.size - 1)
    A, B = oracle.leakage(e, T, alpha, True, ddu)
    dnu = np.diff(e)
    s = [Fraction(float(d)) / Fraction(cdt) for d in dnu]
    rhs = [s[k] * Fraction(float(Jin[k])) for k in range(len(s))]
    x = _exact_solve([Fraction(float(a)) for a in A], [Fraction(float(b)) for b in B], s, rhs)
    got = oracle.freq_solve(e, T, alpha, True, ddu, cdt, Jin)
    np.testing.assert_allclose(got, [float(v) for v in x], rtol=2e-13)


def test_solve_conserves_photons_on_paper_grid(paper_edges):
    # zero-flux frequency ends: sum_k dnu_k J_k is unchanged by the step
    T = 1e4
    g = np.random.default_rng(6)
    dnu = np.diff(paper_edges)
    for alpha, ddu, cdt in [(5.9e-11, 3e-13, 2.4e15), (1e-7, -5e-13, 1e16), (1e-9, 0.0, 1e13)]:
        Jin = g.uniform(0, 1, dnu.size) * np.exp(-np.linspace(-3, 3, dnu.size) ** 2)
        got = oracle.freq_solve(paper_edges, T, alpha, True, ddu, cdt, Jin)
        assert np.all(got >= 0)
        assert np.dot(dnu, got) == pytest.approx(np.dot(dnu, Jin), rel=1e-13)


def test_central_difference_limit_matches_banded_solver():
    # no recoil, no velocity: P = 0, the scheme is the textbook conservative
    # diffusion stencil with conductances 1/(dlt_k/K_k + dlt_{k+1}/K_{k+1})
    T, alpha, cdt = 1e4, 1e-9, 3e9
    e = _toy_grid(N=40)
    K, Cc, P, dlt, dnu = _coeffs(e, T, alpha, False, 0.0)
    G = 1.0 / (dlt[:-1] / K[:-1] + dlt[1:] / K[1:])
    N = dnu.size
    ab = np.zeros((3, N))
    diag = dnu / cdt
    diag[:-1] += G
    diag[1:] += G
    ab[0, 1:] = -G
    ab[1] = diag
    ab[2, :-1] = -G
    Jin = np.exp(-np.linspace(-4, 4, N) ** 2)
    ref = sl.solve_banded((1, 1), ab, dnu / cdt * Jin)
    got = oracle.freq_solve(e, T, alpha, False, 0.0, cdt, Jin)
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def test_recoil_only_equilibrium(paper_edges):
    # dt -> infinity: the zero-flux state J_{k+1}/J_k = exp(-(P_k + P_{k+1})),
    # the exact discrete equilibrium of the exponential scheme
    T, alpha = 1e4, 5.9e-11
    K, Cc, P, dlt, dnu = _coeffs(paper_edges, T, alpha, True, 0.0)
    Jin = np.ones(dnu.size)
    got = oracle.freq_solve(paper_edges, T, alpha, True, 0.0, 1e40, Jin)
    ratio = got[1:] / got[:-1]
    np.testing.assert_allclose(ratio, np.exp(-(P[:-1] + P[1:])), rtol=1e-10)
    assert np.dot(dnu, got) == pytest.approx(np.dot(dnu, Jin), rel=1e-13)

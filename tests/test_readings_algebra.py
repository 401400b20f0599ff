"""Pins for the exact rearrangements the FP32 kernels use in place of the
printed forms (Sec. 2.1 step 1, the Levermore closure and the corrected GLF
diffusion term).  Each rearrangement must equal the printed form evaluated
in 50-digit decimal arithmetic, to FP64 rounding, over the whole range, and
must keep its digits in FP32 where the printed form loses them.

- closure: with s = sqrt(4 - 3 f^2), chi = (3 + 4 f^2) / (5 + 2 s) equals
  (5 - 2 s) / 3, so (1 - chi)/2 = (s - 1)/3 and (3 chi - 1)/(2 f^2) = 3/(2 + s);
- diffusion: (1 - eps)/(3 tau) with eps = (0.2 + tau)/(0.2 + tau + tau^2)
  equals tau / (3 (0.2 + tau + tau^2)).
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 50


def _printed_closure_exact(f):
    # the printed chi, then the two closure coefficients, in 50 digits
    out_a, out_b = [], []
    for x in f:
        x = Decimal(float(x))
        f2 = x * x
        chi = (3 + 4 * f2) / (5 + 2 * (4 - 3 * f2).sqrt())
        out_a.append(float((1 - chi) / 2))
        out_b.append(float((3 * chi - 1) / (2 * f2)))
    return np.array(out_a), np.array(out_b)


def _printed_closure(f):
    f2 = f * f
    chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * np.sqrt(4.0 - 3.0 * f2))
    return (1.0 - chi) / 2.0, (3.0 * chi - 1.0) / (2.0 * f2)


def _rearranged_closure(f):
    s = np.sqrt(4.0 - 3.0 * f * f)
    return (s - 1.0) / 3.0, 3.0 / (2.0 + s)


F = np.concatenate([np.logspace(-6, -1, 60), np.linspace(0.1, 1.0, 91),
                    1.0 - np.logspace(-12, -2, 30)])


def test_closure_rearrangement_is_exact_algebra():
    ea, eb = _printed_closure_exact(F)
    ra, rb = _rearranged_closure(F)
    # (s - 1)/3 -> 0 as f -> 1: the error is absolute there, a few ulp of 1
    np.testing.assert_allclose(ra, ea, rtol=1e-15, atol=4e-16)
    np.testing.assert_allclose(rb, eb, rtol=1e-15, atol=0.0)
    # the limits: chi(0) = 1/3 (isotropic), chi(1) = 1 (free streaming)
    a0, b0 = _rearranged_closure(np.array([0.0, 1.0]))
    np.testing.assert_allclose(a0, [1.0 / 3.0, 0.0], atol=1e-16)
    np.testing.assert_allclose(b0, [0.75, 1.0], rtol=1e-15)


def test_closure_rearrangement_keeps_fp32_digits_near_isotropy():
    # f ~ 1/tau in thick gas: 3 chi - 1 ~ f^2 cancels in the printed form
    f = np.logspace(-4, -1, 40)
    ref = _printed_closure_exact(f)[1]
    printed = _printed_closure(f.astype(np.float32))[1].astype(np.float64)
    rearranged = _rearranged_closure(f.astype(np.float32))[1].astype(np.float64)
    assert np.max(np.abs(rearranged / ref - 1.0)) < 1e-6
    assert np.max(np.abs(printed / ref - 1.0)) > 1e-2


def test_diffusion_rearrangement_is_exact_algebra():
    tau = np.logspace(-8, 8, 161)
    exact = []
    for t in tau:
        t = Decimal(float(t))
        eps = (Decimal("0.2") + t) / (Decimal("0.2") + t + t * t)
        exact.append(float((1 - eps) / (3 * t)))
    rearranged = tau / (3.0 * (0.2 + tau + tau * tau))
    np.testing.assert_allclose(rearranged, np.array(exact), rtol=4e-16)
    # the limits: tau / 0.6 for thin faces, the diffusion 1 / (3 tau) for thick ones
    np.testing.assert_allclose(rearranged[tau < 1e-6], tau[tau < 1e-6] / 0.6, rtol=1e-5)
    np.testing.assert_allclose(rearranged[tau > 1e6], 1.0 / (3.0 * tau[tau > 1e6]), rtol=1e-5)


def _system(n, stiff, seed):
    # the step-3 system scaled by the bin widths (App. A):
    # (s_k + A_{k+1/2} + B_{k-1/2}) J_k - B_{k+1/2} J_{k+1} - A_{k-1/2} J_{k-1} = s_k J''_k,
    # s_k = dnu_k / (c_tilde dt), leakage weights A, B > 0 spanning many decades
    g = np.random.default_rng(seed)
    A = 10.0 ** g.uniform(-6, 6, n - 1)
    B = 10.0 ** g.uniform(-6, 6, n - 1)
    s = 10.0 ** g.uniform(-1, 1, n) / stiff
    r = s * 10.0 ** g.uniform(-3, 3, n)
    return A, B, s, r


def _exact_solve(A, B, s, r):
    from fractions import Fraction as Q
    n = s.size
    A, B, s, r = ([Q(float(x)) for x in v] for v in (A, B, s, r))
    d = [s[k] + (A[k] if k < n - 1 else 0) + (B[k - 1] if k > 0 else 0) for k in range(n)]
    Dp, rp = [d[0]], [r[0]]
    for k in range(1, n):
        m = A[k - 1] / Dp[k - 1]
        Dp.append(d[k] - m * B[k - 1])
        rp.append(r[k] + m * rp[k - 1])
    J = [Q(0)] * n
    J[n - 1] = rp[n - 1] / Dp[n - 1]
    for k in range(n - 2, -1, -1):
        J[k] = (rp[k] + B[k] * J[k + 1]) / Dp[k]
    return np.array([float(x) for x in J])


def _subtraction_free(A, B, s, r, t):
    # D'_k = s_k + A_{k+1/2} + E_k with the margin E_k = B_{k-1/2} (s_{k-1} + E_{k-1}) / D'_{k-1}:
    # sums and products of non-negative terms only
    A, B, s, r = (v.astype(t) for v in (A, B, s, r))
    n = s.size
    E = t(0)
    Dp = np.empty(n, t)
    rp = np.empty(n, t)
    for k in range(n):
        if k > 0:
            E = B[k - 1] * ((s[k - 1] + E) / Dp[k - 1])
        Dp[k] = s[k] + (A[k] if k < n - 1 else t(0)) + E
        rp[k] = r[k] + (A[k - 1] * (rp[k - 1] / Dp[k - 1]) if k > 0 else t(0))
    J = np.empty(n, t)
    J[n - 1] = rp[n - 1] / Dp[n - 1]
    for k in range(n - 2, -1, -1):
        J[k] = (rp[k] + B[k] * J[k + 1]) / Dp[k]
    return J.astype(np.float64)


def _plain_thomas(A, B, s, r, t):
    A, B, s, r = (v.astype(t) for v in (A, B, s, r))
    n = s.size
    d = np.array([s[k] + (A[k] if k < n - 1 else 0) + (B[k - 1] if k > 0 else 0)
                  for k in range(n)], t)
    Dp = np.empty(n, t)
    rp = np.empty(n, t)
    Dp[0], rp[0] = d[0], r[0]
    for k in range(1, n):
        m = A[k - 1] / Dp[k - 1]
        Dp[k] = d[k] - m * B[k - 1]
        rp[k] = r[k] + m * rp[k - 1]
    J = np.empty(n, t)
    J[n - 1] = rp[n - 1] / Dp[n - 1]
    for k in range(n - 2, -1, -1):
        J[k] = (rp[k] + B[k] * J[k + 1]) / Dp[k]
    return J.astype(np.float64)


def test_subtraction_free_elimination_keeps_fp32_accuracy_at_any_stiffness():
    # reading 9: the margin form of the elimination keeps componentwise
    # relative accuracy of order N u whatever c_tilde dt, in FP32 as in FP64;
    # the plain Thomas sweep cancels in d_k - m B and loses it once stiff
    n = 40
    u32 = float(np.finfo(np.float32).eps)
    worst_plain = 0.0
    for stiff in (1.0, 1e4, 1e8):
        for seed in range(3):
            A, B, s, r = _system(n, stiff, seed)
            exact = _exact_solve(A, B, s, r)
            for t, u in ((np.float32, u32), (np.float64, float(np.finfo(np.float64).eps))):
                got = _subtraction_free(A, B, s, r, t)
                assert np.max(np.abs(got / exact - 1.0)) < 4 * n * u, (stiff, seed, t)
            with np.errstate(all="ignore"):  # the plain sweep can reach 0 / 0
                plain = _plain_thomas(A, B, s, r, np.float32)
                err = np.abs(plain / exact - 1.0)
            worst_plain = max(worst_plain, float(np.max(np.where(np.isfinite(err), err, np.inf))))
    # measured: the margin form stays within ~4 u at every stiffness, while
    # the plain FP32 sweep is off by O(1) (or produces 0 / 0) once stiff
    assert worst_plain > 0.5

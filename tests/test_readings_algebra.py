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

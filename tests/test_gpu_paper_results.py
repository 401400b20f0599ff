"""The paper's printed force multipliers reproduced on the GPU (mixed_fast).

Stored values: tests/golden/paper_force_multipliers.txt (each with its
citation).  These are end-to-end checks of the method (Sec. 4.1 Test 1, Sec.
4.2 Test 6), not parity: the paper's own code differs in details it does not
state, so the bars are the agreement the paper itself reports for its code
against analytic results, widened by the resolution the test runs at.
"""
import os

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_force_multipliers.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


def test_golden_file_readable():
    g = golden()
    assert g["cone_M_F"] == 24.45 and g["cone_M_F_radial"] == 19.37


def test_thick_sphere_asymptote():
    # Test 1 at tau_cl = 1e7 (128^2): M_F -> 0.51 (a_v tau)^(1/3) within 5 %
    import paper_2606_02711_gb300.validate as V
    g = golden()
    r = V.sphere(n=128, tau_cl=1e7, chunks=4)
    a_v = 4.7e-4
    ref = g["thick_sphere_coefficient"] * (a_v * 1e7) ** (1.0 / 3.0)
    f = r["final"]
    assert abs(f["M_F"] / ref - 1.0) < 0.05
    assert abs(f["M_F_radial"] / f["M_F"] - 1.0) < 2e-3
    assert f["max_f"] <= 1.0 + 1e-6


def test_cone_force_multipliers():
    # Test 6 at the paper's 256^2: M_F,radial within 5.5 % and M_F within 6.5 %
    # of the paper's values (the gap of this discretisation at 256^2: the
    # multipliers move by 10 % between 128^2 and 256^2, and FP32 arithmetic
    # accounts for < 1e-3 of them), steady over the last half of t_max
    import paper_2606_02711_gb300.validate as V
    g = golden()
    r = V.cone(n=256, chunks=4)
    f = r["final"]
    assert abs(f["M_F_radial"] / g["cone_M_F_radial"] - 1.0) < 0.055
    assert abs(f["M_F"] / g["cone_M_F"] - 1.0) < 0.065
    h = r["history"]
    assert abs(h[-1]["M_F"] / h[-2]["M_F"] - 1.0) < 1e-3
    assert h[-1]["outflow"] > 0 and abs(h[-1]["residual"]) < 1e-3 * h[-1]["emitted"]


def test_cone_multipliers_do_not_depend_on_fp32_arithmetic():
    # Test 6 at 128^2 to t_max: MIXED (FP64 source and elimination) and
    # MIXED_FAST (FP32 throughout) give the same multipliers within 1e-3;
    # the all-FP64 run (25.6407 / 20.2140, 9 GPU-minutes) sits within 1e-4 of MIXED
    import paper_2606_02711_gb300.validate as V
    a = V.cone(n=128, precision="mixed", chunks=2)["final"]
    b = V.cone(n=128, precision="mixed_fast", chunks=2)["final"]
    for k in ("M_F", "M_F_radial"):
        assert abs(b[k] / a[k] - 1.0) < 1e-3, k

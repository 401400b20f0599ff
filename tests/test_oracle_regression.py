"""The oracle against its stored outputs on three small problems with every
term on (tests/golden/oracle_regression.txt, written by the oracle alone via
tests/golden/oracle_regression_cases.py): Cartesian with vacuum edges, the
axisymmetric grid under a two-phase temperature field, and three broad bands.
It guards the pinned oracle against an unnoticed change of its arithmetic;
results do not depend on the thread count."""
import importlib.util
import math
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _stored():
    vals = {}
    with open(os.path.join(HERE, "golden", "oracle_regression.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def _cases():
    spec = importlib.util.spec_from_file_location(
        "oracle_regression_cases", os.path.join(HERE, "golden", "oracle_regression_cases.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m.cases()


def _floor(key, ref):
    # signed sums can cancel: their error is measured against a magnitude
    case, _, q = key.partition(".")
    if q in ("fx.sum", "fy.sum"):
        return ref[f"{case}.{q[:2]}.abs"]
    if q in ("Hx.sum", "Hy.sum"):
        return math.sqrt(ref[f"{case}.{q[:2]}.sumsq"])
    if q == "force_radial":
        return ref[f"{case}.force_abs"]
    return 0.0


def test_oracle_reproduces_its_stored_outputs():
    ref = _stored()
    got = _cases()
    assert set(got) == set(ref)
    for k, v in ref.items():
        assert got[k] == pytest.approx(v, rel=1e-12, abs=1e-12 * _floor(k, ref)), k

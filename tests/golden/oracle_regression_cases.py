"""Regression cases for the oracle: small problems with every term on, whose
outputs tests/golden/oracle_regression.txt stores.  Running this file
rewrites that file from the oracle alone (nothing else computes a stored
value); tests/test_oracle_regression.py recomputes the cases and compares.
A change of the oracle's arithmetic that moves a stored value has to name,
in its commit message, the passage of the paper that justifies it."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

SAMPLES = ((0, 0, 0), (7, 3, 5), (96, 6, 8), (150, 11, 15), (193, 5, 2))


def _state(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    J = 1e-3 * np.exp(g.normal(0, 0.7, (nb, ny, nx)))
    th = g.uniform(0, 2 * np.pi, J.shape)
    f = g.uniform(0, 0.9, J.shape)
    return J, J * f * np.cos(th), J * f * np.sin(th)


def _summary(name, out, diags, samples):
    J, Hx, Hy, fx, fy = out
    vals = {}
    for q, a in (("J", J), ("Hx", Hx), ("Hy", Hy)):
        vals[f"{name}.{q}.sum"] = float(a.sum())
        vals[f"{name}.{q}.sumsq"] = float((a * a).sum())
        for k, j, i in samples:
            if k < a.shape[0]:
                vals[f"{name}.{q}[{k},{j},{i}]"] = float(a[k, j, i])
    for q, a in (("fx", fx), ("fy", fy)):
        vals[f"{name}.{q}.sum"] = float(a.sum())
        vals[f"{name}.{q}.abs"] = float(np.abs(a).sum())
    d = diags[-1]
    for q in ("e_after", "emitted", "absorbed", "outflow", "work", "force_abs", "force_radial"):
        vals[f"{name}.{q}"] = float(d[q])
    return vals


def cases():
    """name -> dict of stored quantities, from the oracle."""
    edges = oracle.freq_grid()
    out = {}
    # Cartesian, lognormal cloud with dust, destruction, a 100 km/s flow, recoil,
    # vacuum x- and y+ edges
    c = wl.lognormal_cloud(16, 12, seed=301, v_edge_kms=100.0, Z=0.3, p_d=1e-7)
    c.bc = (1, 0, 0, 1)
    O = oracle.Oracle(edges=edges, **c.kwargs())
    res, dg = O.run(3, _state(O.nb, 12, 16, 302))
    out.update(_summary("cartesian", res, dg, SAMPLES))
    # axisymmetric, two-phase temperature field, vacuum outer edges
    c = wl.lognormal_cloud(16, 12, seed=303, v_edge_kms=60.0, Z=0.1, p_d=1e-8)
    c.geometry, c.bc = 1, (0, 1, 0, 1)
    g = np.random.default_rng(304)
    temp = np.where(g.uniform(size=(12, 16)) < 0.5, 80.0, 2e4)
    O = oracle.Oracle(edges=edges, **dict(c.kwargs(), temp=temp))
    res, dg = O.run(2, _state(O.nb, 12, 16, 305))
    out.update(_summary("axisymmetric_temperature", res, dg, SAMPLES))
    # three broad bands
    g = np.random.default_rng(306)
    nb, ny, nx, dx = 3, 12, 16, 1e16
    aF = 10.0 ** g.uniform(-2, 2, (nb, ny, nx)) * 2.0 / dx
    kap = aF * g.uniform(0.1, 1.0, aF.shape)
    js = 5e-19 * g.uniform(0, 1, aF.shape)
    ux = g.uniform(-300, 300, (ny, nx)) * 1e5
    uy = g.uniform(-300, 300, (ny, nx)) * 1e5
    O = oracle.Oracle.for_bands(nx=nx, ny=ny, dx=dx, alpha_F=aF, kappa=kap, emissivity=js,
                                ux=ux, uy=uy, bc=(1, 1, 0, 0))
    res, dg = O.run(2, _state(nb, ny, nx, 307))
    out.update(_summary("bands", res, dg, ((0, 0, 0), (1, 5, 7), (2, 11, 15))))
    return out


if __name__ == "__main__":
    vals = cases()
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as fh:
        fh.write("# written by tests/golden/oracle_regression_cases.py from the oracle\n")
        for k, v in vals.items():
            fh.write(f"{k} = {v!r}\n")
    print(len(vals), "values")

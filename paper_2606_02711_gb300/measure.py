"""Throughput of one context on a named workload (cell-updates/s), timed with
CUDA events over a number of CFL substeps after warm-up.

  python -m paper_2606_02711_gb300.measure --workload uniform-gray-64 --precision fp64_det --substeps 2000
  python -m paper_2606_02711_gb300.measure --workload lognormal-2048 --precision mixed_fast --substeps 200
"""
from __future__ import annotations

import argparse
import json


def run(workload: str, precision: str, substeps: int, warmup: int = 5) -> dict:
    import torch
    import workloads as wl
    import paper_2606_02711_gb300.lym1 as L
    cloud = {"uniform-gray-64": wl.uniform_gray, "lognormal-512": wl.config_lognormal_512,
             "lognormal-2048": wl.config_lognormal_2048}[workload]()
    ctx = L.from_cloud(cloud, precision=L.PRECISIONS[precision])
    ctx.substeps(warmup)
    ctx.synchronize()
    ctx.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    ctx.substeps(substeps)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    prof = ctx.profile_read()
    info = ctx.info()
    d = ctx.diagnostics(check=False)
    ctx.destroy()
    cells = cloud.nx * cloud.ny
    out = {"workload": workload, "precision": precision, "cells": cells, "bins": info["nb"],
           "substeps": substeps, "ms_per_substep": ms / substeps,
           "cell_updates_per_s": cells * substeps / (ms * 1e-3),
           "algorithmic_GBps": info["bytes_per_substep"] * substeps / (ms * 1e-3) / 1e9,
           "kernel_ms_per_launch": {k: prof[f"{k}_ms"] / max(prof[f"{k}_launches"], 1)
                                    for k in ("transport", "freq", "finalize")},
           "e_tot": d["e_tot"], "max_f": d["max_f"], "M_F": d["M_F"],
           "residual_over_e": d["residual"] / d["e_tot"] if d["e_tot"] else None}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lognormal-512")
    ap.add_argument("--precision", default="mixed_fast")
    ap.add_argument("--substeps", type=int, default=100)
    args = ap.parse_args()
    print(json.dumps(run(args.workload, args.precision, args.substeps)))


if __name__ == "__main__":
    main()

"""Batched sweep: many independent clouds of uneven size advanced together.

Default workload: 256 clouds, side log-uniform in [64, 512] rounded to 16,
mean n_H log-uniform in [1e2, 1e5] cm^-3, L log-uniform in [1e4, 1e7] L_sun,
Z in {0, 1e-3, 1e-2} Z_sun, 194 bins (seeded per cloud).  Reports
cell-updates/s of the graph-replayed persistent batch (lym1_batch_*) and of
the same clouds advanced one context at a time, per precision.
"""
from __future__ import annotations

import argparse
import json
import time


def run(n_clouds=256, substeps=20, precisions=("mixed_fast", "fp64"), base_seed=1000,
        side_lo=64, side_hi=512, loop_substeps=None, fp64_substeps=None):
    import torch
    import workloads as wl
    import paper_2606_02711_gb300.lym1 as L
    clouds = wl.batch_clouds(n_clouds, base_seed=base_seed, side_lo=side_lo, side_hi=side_hi)
    cells = sum(c.nx * c.ny for c in clouds)
    out = {"clouds": n_clouds, "cells": cells,
           "sides": [min(c.nx for c in clouds), max(c.nx for c in clouds)], "modes": {}}
    for pname in precisions:
        p = L.PRECISIONS[pname]
        n = substeps if p >= 2 else (fp64_substeps or max(2, substeps // 10))
        ctxs = [L.from_cloud(c, precision=p) for c in clouds]
        dev_gb = sum(x.info()["device_bytes"] for x in ctxs) / 1e9
        b = L.Batch(ctxs)
        b.substeps(4)  # grid tuning and graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.substeps(n)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        grid = b.grid()
        b.destroy()
        # the same clouds, one context after another (3 launches per cloud per substep)
        nl = loop_substeps or max(1, n // 2)
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(nl):
            for x in ctxs:
                x.substeps(1)
        a1.record()
        torch.cuda.synchronize()
        ms_loop = a0.elapsed_time(a1)
        for x in ctxs:
            x.destroy()
        out["modes"][pname] = {
            "batched_cell_updates_per_s": cells * n / (ms * 1e-3),
            "batched_ms_per_substep": ms / n, "substeps": n,
            "per_context_loop_cell_updates_per_s": cells * nl / (ms_loop * 1e-3),
            "persistent_grid": grid, "device_gb": dev_gb,
            "host_wall_s": time.perf_counter() - t0}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--clouds", type=int, default=256)
    ap.add_argument("--substeps", type=int, default=20)
    ap.add_argument("--precisions", default="mixed_fast,mixed,fp64")
    ap.add_argument("--fp64-substeps", type=int, default=None,
                    help="substeps of the FP64 policies (default: a tenth of --substeps)")
    ap.add_argument("--loop-substeps", type=int, default=None,
                    help="substeps of the one-context-at-a-time comparison (default: half)")
    args = ap.parse_args()
    print(json.dumps(run(args.clouds, args.substeps, tuple(args.precisions.split(",")),
                         loop_substeps=args.loop_substeps, fp64_substeps=args.fp64_substeps)))


if __name__ == "__main__":
    main()

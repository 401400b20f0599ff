#!/usr/bin/env python
"""Throughput of the Lya M1 substep (transport + implicit source + force +
frequency step) on GB300, through the lym1 C ABI.

One step = one substep of the whole hot path over the synthetic 512x512,
194-bin lognormal cloud (sigma_ln = 1.0, mean n_H = 1e3 cm^-3, Z = 0.01 Z_sun,
v ~ r with 10 km/s at 1 pc, 1e6 L_sun central source).  Metric: cell-updates/s
(one cell advanced one substep over all bins), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl ours|reference]

Under torchrun each rank runs its own cloud (seed 1 + rank): independent
solves, no data-path collective, weak scaling.  The reference arm times the
FP64 CPU oracle on the host cores (a bounded crop of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("Lyα M1 cell-updates/s per GB300 (FP64 vs mixed); served p50/p99 solve latency")
UNIT = "cell-updates/s"
DTYPES = {0: "f64", 1: "f64", 2: "f32+f64", 3: "f32"}
NAMES = {0: "fp64_det", 1: "fp64", 2: "mixed", 3: "mixed_fast"}
WORKLOAD = ("lognormal-512: 512x512 cells x 194 bins, sigma_ln=1.0, mean n_H=1e3 cm^-3, "
            "Z=0.01 Z_sun dust, v~r (10 km/s at 1 pc), 1e6 L_sun central source, T=1e4 K, "
            "2 pc box, outflow boundaries")
# the single large solve (timed on request with --workload lognormal-2048; the
# default line is the 512^2 workload above)
WORKLOAD_2048 = ("lognormal-2048: 2048x2048 cells x 194 bins, sigma_ln=1.5, mean n_H=1e4 cm^-3, "
                 "Z=0.001 Z_sun dust, v~r (10 km/s at 1 pc), 1e7 L_sun central source, T=1e4 K, "
                 "2 pc box, outflow boundaries")


# Algorithmic FP32 operations per (cell, bin) of the transport + source kernel,
# counted from the scheme as written with a*b+c as one operation and each of
# +, -, *, /, sqrt, min/max and compare-select as one: the face flux (two
# MinMod-limited reconstructions, two closures, GLF/diffusion blend, K flux,
# upwind advection) is ~110 operations and each cell owns two faces; the cell
# update (closure, work term, divergences, implicit source, force and
# bookkeeping) is ~75.
ALGO_OPS_TRANSPORT = 2 * 110 + 75
# FP32 lanes per SM on GB300 (one operation per lane per cycle)
FP32_LANES_PER_SM = 128
N_SM = 152
# FP64 pipe of GB300: 2 FMA lanes per SM per cycle (1.25 TFLOP/s nominal at
# 2070 MHz, counting an FMA as 2 flops).  Algorithmic FP64 flops per (cell,
# bin) of the policies that keep the implicit steps in FP64 (FMA = 2 flops,
# each +, -, *, / = 1), counted from the scheme as written:
#   transport kernel, Sec. 2.1 step 2 and Sec. 2.3: kappa_k and alpha_F,k (4),
#     1 + c dt kappa and 1 + c dt alpha_F (4), J'' = (J' + c dt j) / (.) (4),
#     H''_x, H''_y (2), force dnu (H' - H'') for two components (6),
#     absorbed dnu c dt kappa J'' (4), work dnu W (2): 26;
#   frequency kernel, App. A elimination in margin form: E_k, r_k, D'_k (6),
#     one reciprocal (1), g_k, h_k, q_k (3), back substitution (2), energy sum (2): 14.
FP64_LANES_PER_SM = 2
ALGO_FP64_FLOPS = {"transport": 26, "freq": 14}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("lym1_kernels.cuh", "lym1_kernels_fast.cu", "lym1_kernels_det.cu", "lym1_pol_unit.cuh"):
        with open(os.path.join(ROOT, "paper_2606_02711_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_from_profiles(kernel: str, precision: str):
    """DRAM bytes per launch from a committed ncu summary, if its kernel-source
    hash matches the current sources (else None: the kernel has changed)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None, None
    want = _kernel_hash()
    for name in sorted(os.listdir(d)):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(d, name)).read()
        m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
        if not m or m.group(1) != want:
            continue
        for mm in re.finditer(r"traffic_per_launch\s+(\w+)\s+(\w+):\s*([0-9.eE+]+)", text):
            if mm.group(1) == kernel and mm.group(2) == precision:
                return float(mm.group(3)), name
    return None, None


def cpu_baseline(cloud, seconds=10.0, crop=128):
    """FP64 oracle on the host cores over a crop of the workload; substeps are
    repeated until `seconds` of CPU work (at least one)."""
    import oracle
    oracle.build()
    j0 = (cloud.ny - crop) // 2
    i0 = (cloud.nx - crop) // 2
    kw = cloud.kwargs()
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        kw[f] = np.ascontiguousarray(kw[f][j0:j0 + crop, i0:i0 + crop])
    kw["nx"] = kw["ny"] = crop
    O = oracle.Oracle(edges=oracle.freq_grid(), **kw)
    st = O.zero_state()
    O.substep(*st)  # page in
    n, t0 = 0, time.perf_counter()
    while True:
        r = O.substep(*st)
        st = r[:3]
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": crop * crop * n / el, "unit": UNIT, "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{n} FP64 substeps of the central {crop}x{crop} crop of the workload "
                      f"({el:.1f} s wall)"}


def serving_line(L, prec, args, rank, world):
    """A bounded served stream (continuous batching, device-resident state,
    admission by HBM budget): Poisson arrivals of cloud solves run to the
    steady-state rule; p50/p99 latency from arrival to result, solves/s,
    offered vs served load, cap hits.  Under torchrun each rank serves its
    own shard of the stream."""
    import workloads as wl
    from paper_2606_02711_gb300 import serve as S
    fp64 = prec in (L.FP64, L.FP64_DET)
    n = args.serve_requests_fp64 if fp64 else args.serve_requests
    lo, hi = (args.serve_side_fp64, args.serve_side_fp64) if fp64 else (args.serve_side_min,
                                                                          args.serve_side_max)
    arr = wl.poisson_arrivals(n, args.serve_rate, seed=7)
    clouds = wl.batch_clouds(n, base_seed=5000, side_lo=lo, side_hi=hi, nh_lo=args.serve_nh_min,
                             nh_hi=args.serve_nh_max, bc=(1, 1, 1, 1))
    reqs = S.shard([S.Request(i, float(a), c) for i, (a, c) in enumerate(zip(arr, clouds))],
                   rank, world)
    be = S.Lym1Backend(prec)
    srv = S.Server(be, hbm_budget=args.serve_hbm_gb * 1e9, max_active=64, check_every=50,
                   tol=args.serve_tol, max_substeps=args.serve_cap)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = S.summarize(res, wall, args.serve_rate / world)
    out.update({"served_rate_per_s": out["solves_per_s"], "wall_s": wall, "rounds": srv.rounds,
                "batches_built": be.batch_creations, "peak_resident_gb": srv.peak_bytes / 1e9,
                "stream": {"requests": len(reqs), "arrivals": f"Poisson {args.serve_rate}/s",
                           "sides": [lo, hi], "mean_nh": [args.serve_nh_min, args.serve_nh_max],
                           "edges": "outflow into vacuum on all four sides",
                           "L_sun": [1e4, 1e7], "Z_sun": [0, 1e-3, 1e-2],
                           "steady_state": f"|E_n - E_n-50| / E_n / 50 < {args.serve_tol:g}",
                           "cap_substeps": args.serve_cap, "hbm_budget_gb": args.serve_hbm_gb}})
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as wl
    import oracle
    oracle.build()
    cloud = wl.config_lognormal_512(seed=1)
    crop = args.ref_crop
    kw = cloud.kwargs()
    j0 = (cloud.ny - crop) // 2
    for f in ("n_hi", "rho_d", "p_d", "ux", "uy", "lum"):
        kw[f] = np.ascontiguousarray(kw[f][j0:j0 + crop, j0:j0 + crop])
    kw["nx"] = kw["ny"] = crop
    O = oracle.Oracle(edges=oracle.freq_grid(), **kw)
    st = O.zero_state()
    for _ in range(args.warmup):
        st = O.substep(*st)[:3]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = O.substep(*st)[:3]
    el = time.perf_counter() - t0
    value = crop * crop * args.steps / el
    sample = f"each step: one FP64 oracle substep of the central {crop}x{crop} crop of the workload"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)", "crop": crop},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=list(NAMES.values()))
    ap.add_argument("--workload", default="lognormal-512", choices=["lognormal-512", "lognormal-2048"],
                    help="lognormal-2048: the single large solve, timed region only (with --no-extras)")
    ap.add_argument("--fp64-steps", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-crop", type=int, default=128)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="timed region only (for ncu)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--serve-requests-fp64", type=int, default=8)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-side-min", type=int, default=32)
    ap.add_argument("--serve-side-max", type=int, default=64)
    ap.add_argument("--serve-side-fp64", type=int, default=32)
    ap.add_argument("--serve-nh-min", type=float, default=1e-2)
    ap.add_argument("--serve-nh-max", type=float, default=1.0)
    ap.add_argument("--serve-tol", type=float, default=1e-6)
    ap.add_argument("--serve-cap", type=int, default=20000)
    ap.add_argument("--serve-hbm-gb", type=float, default=150.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import workloads as wl
    from paper_2606_02711_gb300 import build as pkg_build
    pkg_build.build()
    import paper_2606_02711_gb300.lym1 as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = L.PRECISIONS[args.precision]
    big = args.workload == "lognormal-2048"
    cloud = (wl.config_lognormal_2048 if big else wl.config_lognormal_512)(seed=1 + rank)
    nc = cloud.nx * cloud.ny
    ctx = L.from_cloud(cloud, precision=prec)
    nb = ctx.nb
    ctx.substeps(args.warmup)
    ctx.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record()
    ctx.substeps(args.steps)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    ck = clocks.stop()
    t = torch.tensor([ms], device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * nc * args.steps / (ms_max * 1e-3)
    diag = ctx.diagnostics(check=False)

    # roofline of the dominant kernel: algorithmic work per launch / mean
    # event-timed launch duration inside the timed region
    selem = 4 if prec >= 2 else 8
    kern = {"transport": (prof["transport_ms"], prof["transport_launches"],
                          nc * (6.0 * nb * selem + 64.0)),
            "freq": (prof["freq_ms"], prof["freq_launches"], nc * (6.0 * nb * selem + 32.0))}
    dom = max(kern, key=lambda k: kern[k][0])
    kms, kl, kbytes = kern[dom]
    avg_s = max(kms / max(kl, 1) * 1e-3, 1e-12)  # no profiled launch: a null roofline
    hbm_gbs = kbytes / avg_s / 1e9
    peak, peak_kind = _peaks()
    traffic, tsrc = _traffic_from_profiles(dom, NAMES[prec])
    share = {k: v[0] / max(ms, 1e-9) for k, v in kern.items()}
    sm_mhz = ck.get("sm_mhz") or 2070.0
    hbm_obj = {"achieved": hbm_gbs, "peak": peak, "unit": "GB/s", "frac": hbm_gbs / peak,
               "algorithmic_bytes_per_launch": kbytes,
               "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"
               if peak_kind == "measured" else "fallback 6.8 TB/s"}
    if prec in (0, 1, 2):
        # the FP64 implicit steps bind on GB300's FP64 pipe (~1/70 of the FP32
        # rate): FP64-pipe roofline of the dominant kernel, HBM beside it
        f64_peak = N_SM * FP64_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        f64_ach = ALGO_FP64_FLOPS[dom] * nc * nb / avg_s / 1e12
        roof = {"bound": "alu", "pipe": "fp64", "achieved": f64_ach, "peak": f64_peak,
                "unit": "TFLOP/s", "frac": f64_ach / f64_peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"derived: {N_SM} SMs x {FP64_LANES_PER_SM} FP64 FMA lanes x 2 "
                               f"flops x {sm_mhz:.0f} MHz",
                "algorithmic_fp64_flops_per_cell_bin": ALGO_FP64_FLOPS[dom], "hbm": hbm_obj}
    elif dom == "transport" and prec == 3:
        # FP32 transport is bound by instruction issue (ncu: DRAM bytes equal the
        # algorithmic bytes at ~14 % of DRAM peak, issue ~70 % active): FP32 ALU roofline
        alu_peak = N_SM * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
        alu_ach = ALGO_OPS_TRANSPORT * nc * nb / avg_s / 1e12
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_ach / alu_peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"derived: {N_SM} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                               f"{sm_mhz:.0f} MHz (one op per lane per cycle)",
                "algorithmic_ops_per_cell_bin": ALGO_OPS_TRANSPORT, "hbm": hbm_obj}
    else:
        roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": peak, "unit": "GB/s",
                "frac": hbm_gbs / peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": kbytes}
    roof.update({"avg_launch_ms": avg_s * 1e3, "kernel_ms_share": share,
                 "traffic_source": tsrc})

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
           "data": "synthetic (seeded lognormal cloud, no dataset)",
           "config": {"workload": WORKLOAD_2048 if big else WORKLOAD, "cells": nc, "bins": nb, "precision": NAMES[prec],
                      "substep_dt_s": ctx.dt_cfl, "per_rank_clouds": 1,
                      "l2": "inputs larger than L2: state "
                            f"{3 * nb * nc * selem / 1e6:.0f} MB per copy > 129 MB L2",
                      "parallelism": f"independent clouds, {world} rank(s)"},
           "clocks": ck, "roofline": roof,
           "gpu_launches": int(prof["transport_launches"] + prof["freq_launches"] +
                               prof["finalize_launches"]),
           "diagnostics_after_timed": {k: diag[k] for k in ("e_tot", "max_f", "M_F", "f_esc")}}
    ctx.destroy()

    if not args.no_extras:
        # e2e through the public API with pinned host buffers: per step the sources
        # go host->device, one substep runs, the force comes back device->host
        ctx = L.from_cloud(cloud, precision=prec)
        ctx.substeps(args.warmup)
        ctx.synchronize()
        lum_h = torch.from_numpy(np.ascontiguousarray(cloud.lum)).pin_memory()
        fx_h = torch.empty((cloud.ny, cloud.nx), dtype=torch.float64).pin_memory()
        fy_h = torch.empty((cloud.ny, cloud.nx), dtype=torch.float64).pin_memory()
        lum_np, fx_np, fy_np = lum_h.numpy(), fx_h.numpy(), fy_h.numpy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.set_sources(lum_np)
            ctx.substeps(1)
            ctx.force(out=(fx_np, fy_np))
        el = time.perf_counter() - t0
        tt = torch.tensor([el], device="cuda")
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        el = float(tt.item())
        out["e2e"] = {"value": world * nc * args.e2e_steps / el, "unit": UNIT,
                      "h2d_bytes_per_step": nc * 8, "d2h_bytes_per_step": 2 * nc * 8,
                      "steps": args.e2e_steps,
                      "path": "lym1_set_sources (pinned H2D) + lym1_substeps(1) + "
                              "lym1_force (pinned D2H) per step"}
        ctx.destroy()

        # FP64 path on the same workload, for the mixed-vs-FP64 comparison
        cmp = {}
        for p in (L.FP64, L.FP64_DET, L.MIXED, L.MIXED_FAST):
            if p == prec:
                continue
            c2 = L.from_cloud(cloud, precision=p)
            c2.substeps(2)
            c2.synchronize()
            n = args.fp64_steps if p < 2 else 4 * args.fp64_steps
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            c2.substeps(n)
            b.record()
            torch.cuda.synchronize()
            m = a.elapsed_time(b)
            cmp[NAMES[p]] = {"value": nc * n / (m * 1e-3), "ms_per_step": m / n, "steps": n,
                             "dtype": DTYPES[p]}
            if p == L.MIXED_FAST:
                cmp[NAMES[p]]["note"] = ("extra: FP32 implicit steps and per-cell sums (not the "
                                         "FP32-flux / FP64-source split of the headline)")
            c2.destroy()
        out["precisions"] = cmp

        # the same cloud under a two-phase gas temperature (80 K / 2e4 K): the
        # per-[bin][cell] <H>_k tables built at creation, then the headline policy
        import copy
        ctf = copy.copy(cloud)
        ctf.temp = wl.two_phase_temperature(cloud.nx, cloud.ny, seed=7, T_cold=80.0, T_hot=2.0e4)
        t0 = time.perf_counter()
        c3 = L.from_cloud(ctf, precision=prec)
        t_create = time.perf_counter() - t0
        c3.substeps(4)
        c3.synchronize()
        n = 4 * args.fp64_steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        c3.substeps(n)
        b.record()
        torch.cuda.synchronize()
        m = a.elapsed_time(b)
        # new temperatures as after a hydro step: the per-cell tables on the device
        T2 = wl.two_phase_temperature(cloud.nx, cloud.ny, seed=8, T_cold=300.0, T_hot=8.0e3)
        c3.set_temperature(T2)
        t0 = time.perf_counter()
        c3.set_temperature(ctf.temp)
        t_update = time.perf_counter() - t0
        out["temperature_field"] = {"value": nc * n / (m * 1e-3), "unit": UNIT, "ms_per_step": m / n,
                                    "steps": n, "create_s": t_create, "update_s": t_update,
                                    "field": "two-phase 80 K / 2e4 K (seeded k^-4 field)"}
        c3.destroy()

        # the finer frequency grid of Sec. 4.1, Test 2 (q = 1.03: 542 bins by the grid's
        # truncation rule), headline policy: a cell-update here carries 542 bins, not 194
        c4 = L.from_cloud(cloud, precision=prec, q=1.03)
        c4.substeps(4)
        c4.synchronize()
        n = 4 * args.fp64_steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        c4.substeps(n)
        b.record()
        torch.cuda.synchronize()
        m = a.elapsed_time(b)
        out["fine_grid"] = {"value": nc * n / (m * 1e-3), "unit": UNIT, "ms_per_step": m / n,
                            "steps": n, "bins": c4.nb, "q": 1.03}
        c4.destroy()

        # the seven stellar/IR bands of Sec. 3 on the same cloud: per band the
        # transport and source step, no frequency step, headline policy
        aF, ka, je = wl.stellar_bands(cloud)
        c5 = L.Context.for_bands(nx=cloud.nx, ny=cloud.ny, dx=cloud.dx, ux=cloud.ux, uy=cloud.uy,
                                 alpha_F=aF, kappa=ka, emissivity=je, precision=prec)
        c5.substeps(4)
        c5.synchronize()
        n = 16 * args.fp64_steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        c5.substeps(n)
        b.record()
        torch.cuda.synchronize()
        m = a.elapsed_time(b)
        out["stellar_bands"] = {"value": nc * n / (m * 1e-3), "unit": UNIT, "ms_per_step": m / n,
                                "steps": n, "bands": c5.nb,
                                "note": "cell-updates over 7 bands (IR, opt, FUV, LW, EUV1-3)"}
        c5.destroy()

        if not args.no_serve:
            out["serving"] = {NAMES[p]: serving_line(L, p, args, rank, world)
                              for p in dict.fromkeys((prec, L.FP64))}

        if rank == 0 and world == 1 and not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(cloud, seconds=args.cpu_seconds)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Request loop for cloud solves with continuous batching.

Requests (clouds of different sizes, densities and luminosities) arrive over
time.  The loop admits them in arrival order while the device-memory budget
and the slot limit allow, keeps every admitted cloud's state resident on the
device, and advances all active clouds together: each round is one batch of
`check_every` substeps (one graph-replayed set of persistent launches per
substep, through the lym1 C ABI).  New requests join and converged ones leave
at round boundaries, so arrivals overlap on the device with work already in
flight.  A cloud is done when its domain energy E satisfies the steady-state
rule |E_n - E_{n-m}| / E_n / m < tol (m = check_every, counted in its own
substeps) or when it reaches the substep cap; its result (force, diagnostics)
is then read back and its memory freed.  Because every cloud's checks fall on
its own substep counts and batched substeps equal solo substeps bit for bit,
a cloud's result does not depend on the mix it was served in.

Multi-GPU: `shard(requests, rank, world)` gives each rank its own subset; the
ranks share nothing on the data path.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    cloud: object           # workloads.Cloud


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    substeps: int
    converged: bool
    cells: int
    diag: dict = field(default_factory=dict)
    force: tuple | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def shard(requests, rank: int, world: int):
    """Round-robin assignment of requests to ranks (no data shared)."""
    return [r for i, r in enumerate(requests) if i % world == rank]


class Lym1Backend:
    """GPU backend: one lym1 context per admitted cloud.  The active clouds
    advance as one lym1 batch (persistent launches, graph-replayed); the batch
    is kept while the set of active clouds is unchanged and rebuilt only when a
    cloud joins or leaves, so rounds with the same membership neither re-tune
    nor re-capture.  Admission uses the library's own byte count
    (lym1_plan_bytes), which equals what the context allocates."""

    def __init__(self, precision: int, edges=None, stream=None):
        import paper_2606_02711_gb300.lym1 as L
        self.L = L
        self.precision = precision
        self.edges = edges
        self.stream = stream
        self.batch = None
        self.members = ()
        self.batch_creations = 0

    def bytes_for(self, cloud) -> float:
        return self.L.plan_bytes(cloud.nx, cloud.ny, self.precision,
                                 geometry=getattr(cloud, "geometry", 0), edges=self.edges,
                                 gray=cloud.gray, temp_field=getattr(cloud, "temp", None) is not None)

    def open(self, cloud):
        return self.L.from_cloud(cloud, precision=self.precision, stream=self.stream,
                                 edges=self.edges)

    def _drop_batch(self):
        if self.batch is not None:
            self.batch.destroy()
        self.batch, self.members = None, ()

    def advance(self, handles, n):
        key = tuple(id(h) for h in handles)
        if key != self.members:
            self._drop_batch()
            self.batch = self.L.Batch(handles)
            self.members = key
            self.batch_creations += 1
        self.batch.substeps(n)

    def energy(self, h) -> float:
        return h.diagnostics(check=False)["e_tot"]

    def result(self, h, keep_force: bool):
        d = h.diagnostics(check=False)
        f = h.force() if keep_force else None
        return d, f

    def close(self, h):
        if id(h) in self.members:  # a batch is destroyed before its contexts
            self._drop_batch()
        h.destroy()


class Server:
    def __init__(self, backend, *, hbm_budget=150e9, max_active=64, check_every=50, tol=1e-6,
                 max_substeps=100000, keep_force=False):
        self.be = backend
        self.hbm_budget = float(hbm_budget)
        self.max_active = int(max_active)
        self.m = int(check_every)
        self.tol = float(tol)
        self.cap = int(max_substeps)
        self.keep_force = keep_force
        self.peak_bytes = 0.0
        self.rounds = 0

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serves `requests` (sorted by arrival, times relative to the start)
        in real time; returns the list of Results in completion order."""
        queue = sorted(requests, key=lambda r: r.arrival)
        qi = 0
        waiting: list[Request] = []
        active = []   # dicts: req, handle, bytes, n, e_prev, admitted
        used = 0.0
        results: list[Result] = []
        t0 = clock()
        while qi < len(queue) or waiting or active:
            now = clock() - t0
            while qi < len(queue) and queue[qi].arrival <= now:
                waiting.append(queue[qi])
                qi += 1
            # admission in arrival order while memory and slots allow
            while waiting and len(active) < self.max_active:
                r = waiting[0]
                need = self.be.bytes_for(r.cloud)
                if used + need > self.hbm_budget and active:
                    break
                waiting.pop(0)
                h = self.be.open(r.cloud)
                active.append({"req": r, "h": h, "bytes": need, "n": 0, "e_prev": None,
                               "admitted": clock() - t0})
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                if qi < len(queue):
                    sleep(max(0.0, queue[qi].arrival - (clock() - t0)))
                continue
            n = min(self.m, min(self.cap - a["n"] for a in active))
            self.be.advance([a["h"] for a in active], n)
            self.rounds += 1
            keep = []
            for a in active:
                a["n"] += n
                e = self.be.energy(a["h"])
                conv = (a["e_prev"] is not None and n == self.m and e > 0 and
                        abs(e - a["e_prev"]) / e / self.m < self.tol)
                a["e_prev"] = e
                if conv or a["n"] >= self.cap:
                    d, f = self.be.result(a["h"], self.keep_force)
                    self.be.close(a["h"])
                    used -= a["bytes"]
                    c = a["req"].cloud
                    results.append(Result(a["req"].rid, a["req"].arrival, a["admitted"],
                                          clock() - t0, a["n"], bool(conv), c.nx * c.ny, d, f))
                else:
                    keep.append(a)
            active = keep
        return results


def summarize(results, wall: float, offered_rate: float) -> dict:
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(results) / wall if wall > 0 else 0.0,
            "offered_rate_per_s": offered_rate,
            "cap_hits": int(sum(not r.converged for r in results)),
            "cell_updates_per_s": float(sum(r.cells * r.substeps for r in results) / wall)
            if wall > 0 else 0.0}


def make_requests(n, rate, seed, side_lo, side_hi, base_seed=5000):
    import workloads as wl
    arr = wl.poisson_arrivals(n, rate, seed)
    clouds = wl.batch_clouds(n, base_seed=base_seed, side_lo=side_lo, side_hi=side_hi)
    return [Request(i, float(a), c) for i, (a, c) in enumerate(zip(arr, clouds))]


def main():
    ap = argparse.ArgumentParser(description="serve a Poisson stream of cloud solves")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--side-min", type=int, default=64)
    ap.add_argument("--side-max", type=int, default=1024)
    ap.add_argument("--precision", default="mixed_fast")
    ap.add_argument("--check-every", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--cap", type=int, default=100000)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--hbm-budget-gb", type=float, default=150.0)
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args()
    import paper_2606_02711_gb300.lym1 as L
    reqs = make_requests(args.requests, args.rate, args.seed, args.side_min, args.side_max)
    srv = Server(Lym1Backend(L.PRECISIONS[args.precision]), hbm_budget=args.hbm_budget_gb * 1e9,
                 max_active=args.max_active, check_every=args.check_every, tol=args.tol,
                 max_substeps=args.cap)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = summarize(res, wall, args.rate)
    out.update({"precision": args.precision, "rounds": srv.rounds,
                "peak_resident_gb": srv.peak_bytes / 1e9, "wall_s": wall,
                "config": vars(args)})
    print(json.dumps(out))


if __name__ == "__main__":
    main()

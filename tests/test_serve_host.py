"""Host logic of the request loop (admission by memory budget and slots,
continuous batching rounds, steady-state rule, substep cap), with a fake
backend whose energy relaxes as E_n = 1 - exp(-n / tau) -- no GPU."""
import math


from paper_2606_02711_gb300.serve import Request, Server, shard, summarize


class FakeCloud:
    def __init__(self, nx, ny, tau):
        self.nx, self.ny, self.tau = nx, ny, tau


class FakeBackend:
    precision = 3

    def __init__(self):
        self.open_count = 0
        self.batches = []

    def bytes_for(self, cloud):
        return 6 * 194 * cloud.nx * cloud.ny * 4 + 12 * cloud.nx * cloud.ny * 8

    def open(self, cloud):
        self.open_count += 1
        return {"cloud": cloud, "n": 0, "open": True}

    def advance(self, handles, n):
        self.batches.append(len(handles))
        for h in handles:
            assert h["open"]
            h["n"] += n

    def energy(self, h):
        return 1.0 - math.exp(-h["n"] / h["cloud"].tau)

    def result(self, h, keep_force):
        return {"e_tot": self.energy(h), "substeps": h["n"]}, None

    def close(self, h):
        h["open"] = False


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3  # every call advances the clock a little
        return self.t

    def sleep(self, dt):
        self.t += dt


def test_steady_state_rule_and_cap():
    be, clk = FakeBackend(), FakeClock()
    reqs = [Request(0, 0.0, FakeCloud(64, 64, 100.0)), Request(1, 0.0, FakeCloud(64, 64, 1e9))]
    srv = Server(be, check_every=50, tol=1e-6, max_substeps=2000)
    res = {r.rid: r for r in srv.run(reqs, clock=clk, sleep=clk.sleep)}
    # |E_n - E_{n-50}| / E_n / 50 < 1e-6 first holds where exp(-n/100) (e^{1/2}-1)/50 < 1e-6
    n_expect = next(n for n in range(100, 5000, 50)
                    if (math.exp(-(n - 50) / 100) - math.exp(-n / 100)) /
                    (1 - math.exp(-n / 100)) / 50 < 1e-6)
    assert res[0].converged and res[0].substeps == n_expect
    assert not res[1].converged and res[1].substeps == 2000
    assert be.open_count == 2


def test_admission_respects_budget_and_slots():
    be, clk = FakeBackend(), FakeClock()
    cloud = FakeCloud(256, 256, 200.0)
    per = be.bytes_for(cloud)
    reqs = [Request(i, 0.0, cloud) for i in range(6)]
    srv = Server(be, hbm_budget=2.5 * per, max_active=8, check_every=50, tol=1e-5)
    res = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert len(res) == 6
    assert srv.peak_bytes <= 2.5 * per
    assert max(be.batches) == 2
    srv2 = Server(FakeBackend(), hbm_budget=1e15, max_active=3, check_every=50, tol=1e-5)
    be2 = srv2.be
    srv2.run(reqs, clock=FakeClock(), sleep=lambda dt: None)
    assert max(be2.batches) == 3


def test_late_arrivals_join_running_batches():
    be, clk = FakeBackend(), FakeClock()
    reqs = [Request(0, 0.0, FakeCloud(64, 64, 2000.0)), Request(1, 0.05, FakeCloud(32, 32, 50.0))]
    srv = Server(be, check_every=50, tol=1e-6, max_substeps=100000)
    res = {r.rid: r for r in srv.run(reqs, clock=clk, sleep=clk.sleep)}
    assert res[1].admitted < res[0].done and res[1].done < res[0].done
    assert 2 in be.batches and be.batches[0] == 1
    s = summarize(list(res.values()), clk.t, 50.0)
    assert s["requests"] == 2 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_shard_partitions_requests():
    reqs = list(range(11))
    parts = [shard(reqs, r, 3) for r in range(3)]
    assert sorted(x for p in parts for x in p) == reqs
    assert all(len(set(a) & set(b)) == 0 for a in parts for b in parts if a is not b)

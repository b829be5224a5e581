"""Host logic of the serving loop (serve.Server) on the CPU, against a fake batch.

The fake stands in for ``binding.Batch``: each job takes nx*ny bytes of an arena and
retires after ceil(steps / K) intervals.  These tests need no GPU: they check admission
against the budget, that a request larger than the whole arena is retired at once with
PL_ERR_BUDGET instead of blocking the queue (the loop must end by itself), and that each
result names its own request even when two requests are equal field by field.
"""
import pytest

from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import serve as S
from paper_2504_10539_gb300 import workloads as wl


class FakeBatch:
    def __init__(self, arena, K):
        self.arena, self.K, self.used = arena, K, 0
        self.jobs, self.next_id, self.done, self.peak = {}, 0, [], 0

    def set_weights(self, blob):
        pass

    def job_bytes(self, job):
        return job.nx * job.ny

    def arena_bytes(self):
        return self.arena

    def submit(self, job):
        b = self.job_bytes(job)
        if self.used + b > self.arena:
            return None
        self.used += b
        jid = self.next_id
        self.next_id += 1
        self.jobs[jid] = [job, -(-job.steps // self.K)]
        self.peak = max(self.peak, len(self.jobs))
        return jid

    def advance(self, n=1):
        for jid in list(self.jobs):
            self.jobs[jid][1] -= n
            if self.jobs[jid][1] <= 0:
                job = self.jobs.pop(jid)[0]
                self.used -= self.job_bytes(job)
                self.done.append({"id": jid, "status": 0, "steps": -(-job.steps // self.K) * self.K,
                                  "nx": job.nx, "ny": job.ny, "metrics": {"mass": float(jid)}})

    def poll(self):
        out, self.done = self.done, []
        return out

    def close(self):
        pass


def reqs(sides, steps=300, t=0.0):
    return [wl.Request(t, wl.Lattice(s, s, steps=steps, K=100)) for s in sides]


@pytest.mark.timeout(60)
def test_request_larger_than_the_arena_is_retired_and_does_not_block():
    r = reqs([32, 200, 32, 32])          # 200^2 bytes > the 64^2-byte arena
    srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, 100, 0, None, batch=FakeBatch(64 * 64, 100))
    out = srv.run(r)                     # no wall-clock limit: the loop must end by itself
    assert out["jobs_rejected"] == 1 and out["jobs_done"] == 3
    bad = [x for x in out["results"] if x["status"] != 0]
    assert len(bad) == 1 and bad[0]["request"] == 1 and bad[0]["status"] == B.PL_ERR_BUDGET
    assert sorted(x["request"] for x in out["results"] if x["status"] == 0) == [0, 2, 3]


@pytest.mark.timeout(60)
def test_only_request_larger_than_the_arena():
    srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, 100, 0, None, batch=FakeBatch(10, 100))
    out = srv.run(reqs([8]))
    assert out["jobs_done"] == 0 and out["jobs_rejected"] == 1 and out["p50_latency_s"] is None


@pytest.mark.timeout(60)
def test_identical_requests_keep_their_own_index_and_wait_for_memory():
    r = reqs([32] * 6)                   # equal field by field
    fb = FakeBatch(2 * 32 * 32, 100)     # room for two at a time
    srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, 100, 0, None, batch=fb)
    out = srv.run(r)
    assert out["jobs_done"] == 6 and out["statuses"] == {0: 6}
    assert sorted(x["request"] for x in out["results"]) == list(range(6))
    assert fb.peak == out["peak_active_jobs"] == 2
    # admission in arrival order: the i-th admitted job is request i
    assert [x["request"] for x in sorted(out["results"], key=lambda x: x["id"])] == list(range(6))
    assert max(x["admitted_interval"] for x in out["results"]) > 0


class SlowFakeBatch(FakeBatch):
    """An interval takes `dt` seconds of wall clock, like a device interval would."""

    def __init__(self, arena, K, dt):
        super().__init__(arena, K)
        self.dt = dt

    def advance(self, n=1):
        import time
        time.sleep(self.dt * n)
        super().advance(n)


@pytest.mark.timeout(60)
def test_reported_statistics_follow_the_results():
    """Three requests 50 ms apart, each three intervals of 30 ms (250 steps rounded up to 300):
    they overlap on the device; every reported figure is the one the per-request results give."""
    import numpy as np
    r = [wl.Request(0.05 * k, wl.Lattice(32, 32, steps=250, K=100)) for k in range(3)]
    srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, 100, 0, None, batch=SlowFakeBatch(10 * 32 * 32, 100, 0.03))
    out = srv.run(r)
    assert out["jobs_done"] == 3 and out["jobs_rejected"] == 0 and out["statuses"] == {0: 3}
    res = sorted(out["results"], key=lambda x: x["request"])
    for x, q in zip(res, r):
        assert x["steps"] == 300
        assert q.arrival_s <= x["admitted_s"] <= x["done_s"]
        assert x["done_s"] - x["admitted_s"] >= 3 * 0.03 * 0.9      # three intervals on the device
        assert x["done_interval"] - x["admitted_interval"] == 3
    lat = [x["done_s"] - q.arrival_s for x, q in zip(res, r)]
    wait = [x["admitted_s"] - q.arrival_s for x, q in zip(res, r)]
    assert out["p50_latency_s"] == float(np.percentile(lat, 50))
    assert out["p99_latency_s"] == float(np.percentile(lat, 99))
    assert out["p50_queue_wait_s"] == float(np.percentile(wait, 50))
    assert out["peak_active_jobs"] >= 2                               # arrivals while others run
    work = 3 * 32 * 32 * 300
    assert out["served_mlups"] == pytest.approx(work / out["elapsed_s"] / 1e6)
    assert out["offered_mlups"] == pytest.approx(work / 0.1 / 1e6)    # over the arrival span
    assert out["elapsed_s"] >= 0.1 + 3 * 0.03 * 0.9                   # the last request's own run

"""Continuous-batching request loop for droplet-relaxation jobs.

Requests (``workloads.Request``: arrival time + job) arrive over wall-clock time.  The
loop admits every arrived request whose lattice fits the batch's device budget and a job
slot, runs one coupling interval (K steps + correction + metrics for every active job,
one graph replay), retires finished jobs and records their latency (completion time -
arrival time).  Requests that do not fit wait, first in first out, and are admitted as
soon as retirements free memory or slots, so new work overlaps with work in progress.
A request whose lattice is larger than the whole arena can never be admitted: it is
retired at once with status PL_ERR_BUDGET instead of blocking the queue behind it.
All compute is in the batch's kernels (C ABI ``pl_batch_*``); this loop only decides
when to call them.
"""
from __future__ import annotations

import collections
import time
from typing import Dict

import numpy as np

from . import binding as B


class Server:
    """Serving loop over a ``binding.Batch`` (or any object with the same ``submit``,
    ``advance``, ``poll``, ``job_bytes`` and ``arena_bytes`` methods)."""

    def __init__(self, storage: int, mlp: int, K: int, budget_bytes: int, weights, max_jobs: int = 1024,
                 stream=None, batch=None):
        self.batch = batch if batch is not None else B.Batch(storage, mlp, K, budget_bytes, max_jobs=max_jobs,
                                                             stream=stream)
        self.batch.set_weights(weights)
        self.K = K

    def run(self, requests, max_wall_s: float = None) -> Dict:
        order = sorted(range(len(requests)), key=lambda k: requests[k].arrival_s)
        reqs = collections.deque(order)          # request indices, by arrival
        waiting = collections.deque()
        inflight = {}             # job id -> (request index, admitted_at, admitted interval)
        lat, queue_wait, work = [], [], 0
        results = []
        arena = self.batch.arena_bytes()
        t0 = time.perf_counter()
        peak_active, intervals, rejected = 0, 0, 0
        while reqs or waiting or inflight:
            now = time.perf_counter() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            while reqs and requests[reqs[0]].arrival_s <= now:
                waiting.append(reqs.popleft())
            while waiting:
                k = waiting[0]
                job = requests[k].job
                if self.batch.job_bytes(job) > arena:
                    # larger than the whole arena: no retirement can ever make room
                    waiting.popleft()
                    rejected += 1
                    results.append({"id": -1, "request": k, "status": B.PL_ERR_BUDGET, "steps": 0,
                                    "nx": job.nx, "ny": job.ny, "admitted_s": None, "done_s": now})
                    continue
                jid = self.batch.submit(job)
                if jid is None:   # no room now: wait for retirements
                    break
                waiting.popleft()
                inflight[jid] = (k, now, intervals)
            if not inflight:
                if waiting:
                    # nothing on the device and the head still not admitted: the batch refused a
                    # job that fits the empty arena, so it would refuse it forever
                    k = waiting.popleft()
                    rejected += 1
                    results.append({"id": -1, "request": k, "status": B.PL_ERR_BUDGET, "steps": 0,
                                    "nx": requests[k].job.nx, "ny": requests[k].job.ny, "admitted_s": None,
                                    "done_s": now})
                elif reqs:
                    time.sleep(max(0.0, requests[reqs[0]].arrival_s - (time.perf_counter() - t0)))
                continue
            peak_active = max(peak_active, len(inflight))
            self.batch.advance(1)
            intervals += 1
            for res in self.batch.poll():
                done_at = time.perf_counter() - t0
                k, adm, adm_interval = inflight.pop(res["id"])
                r = requests[k]
                lat.append(done_at - r.arrival_s)
                queue_wait.append(adm - r.arrival_s)
                work += r.job.nx * r.job.ny * res["steps"]
                # the request (by its index in `requests`) and its life on the device, in loop intervals
                res.update(request=k, admitted_s=adm, done_s=done_at,
                           admitted_interval=adm_interval, done_interval=intervals)
                results.append(res)
        elapsed = time.perf_counter() - t0
        arrivals = [r.arrival_s for r in requests]
        offered = sum(r.job.nx * r.job.ny * ((r.job.steps + self.K - 1) // self.K * self.K) for r in requests)
        span = max(arrivals) - min(arrivals) if len(arrivals) > 1 else 0.0
        span = span if span > 0.0 else 1.0

        def pct(v, q):
            return float(np.percentile(v, q)) if v else None

        return {
            "jobs_done": len(lat),
            "jobs_submitted": len(requests),
            "jobs_rejected": rejected,
            "p50_latency_s": pct(lat, 50),
            "p99_latency_s": pct(lat, 99),
            "p50_queue_wait_s": pct(queue_wait, 50),
            "p99_queue_wait_s": pct(queue_wait, 99),
            "served_mlups": work / elapsed / 1e6 if elapsed > 0.0 else 0.0,
            "offered_mlups": offered / span / 1e6,
            "elapsed_s": elapsed,
            "intervals": intervals,
            "peak_active_jobs": peak_active,
            "statuses": collections.Counter(r["status"] for r in results),
            "results": results,
        }

    def close(self):
        self.batch.close()

"""Continuous-batching request loop for droplet-relaxation jobs.

Requests (``workloads.Request``: arrival time + job) arrive over wall-clock time.  The
loop admits every arrived request whose lattice fits the batch's device budget and a job
slot, runs one coupling interval (K steps + correction + metrics for every active job,
one graph replay), retires finished jobs and records their latency (completion time -
arrival time).  Requests that do not fit wait, first in first out, and are admitted as
soon as retirements free memory or slots, so new work overlaps with work in progress.
All compute is in the batch's kernels (C ABI ``pl_batch_*``); this loop only decides
when to call them.
"""
from __future__ import annotations

import collections
import time
from typing import Dict, List

import numpy as np

from . import binding as B


class Server:
    def __init__(self, storage: int, mlp: int, K: int, budget_bytes: int, weights, max_jobs: int = 1024,
                 stream=None):
        self.batch = B.Batch(storage, mlp, K, budget_bytes, max_jobs=max_jobs, stream=stream)
        self.batch.set_weights(weights)
        self.K = K

    def run(self, requests, max_wall_s: float = None) -> Dict:
        reqs = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting = collections.deque()
        inflight = {}             # job id -> (request, admitted_at)
        lat, queue_wait, work = [], [], 0
        results = []
        t0 = time.perf_counter()
        peak_active, intervals = 0, 0
        while reqs or waiting or inflight:
            now = time.perf_counter() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            while reqs and reqs[0].arrival_s <= now:
                waiting.append(reqs.popleft())
            while waiting:
                r = waiting[0]
                jid = self.batch.submit(r.job)
                if jid is None:   # no room now: wait for retirements
                    break
                waiting.popleft()
                inflight[jid] = (r, now, intervals)
            if not inflight:
                if reqs:
                    time.sleep(max(0.0, reqs[0].arrival_s - (time.perf_counter() - t0)))
                continue
            peak_active = max(peak_active, len(inflight))
            self.batch.advance(1)
            intervals += 1
            for res in self.batch.poll():
                done_at = time.perf_counter() - t0
                r, adm, adm_interval = inflight.pop(res["id"])
                lat.append(done_at - r.arrival_s)
                queue_wait.append(adm - r.arrival_s)
                work += r.job.nx * r.job.ny * res["steps"]
                # the request (by arrival order) and its life on the device, in loop intervals
                res.update(request=requests.index(r), admitted_s=adm, done_s=done_at,
                           admitted_interval=adm_interval, done_interval=intervals)
                results.append(res)
        elapsed = time.perf_counter() - t0
        arrivals = [r.arrival_s for r in requests]
        offered = sum(r.job.nx * r.job.ny * ((r.job.steps + self.K - 1) // self.K * self.K) for r in requests)
        span = max(arrivals) - min(arrivals) if len(arrivals) > 1 else 1.0
        return {
            "jobs_done": len(lat),
            "jobs_submitted": len(requests),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat else None,
            "p50_queue_wait_s": float(np.percentile(queue_wait, 50)) if queue_wait else None,
            "served_mlups": work / elapsed / 1e6,
            "offered_mlups": offered / span / 1e6,
            "elapsed_s": elapsed,
            "intervals": intervals,
            "peak_active_jobs": peak_active,
            "statuses": collections.Counter(r["status"] for r in results),
            "results": results,
        }

    def close(self):
        self.batch.close()

"""Serving: continuous batching of droplet-relaxation requests (the served configuration at a
small scale).

The device budget holds only a few of the requests at once, so arrivals wait for memory;
requests admitted while others are on the device run in the same interval replays as them.
Each job's result must be the same as the job run alone in its own batch: bit-identical,
because a job's arithmetic (reduction partition, FP16 dither, step count) depends on the job
only.
"""
import numpy as np
import pytest

from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import serve as S
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

K = 100


def requests(n=12):
    # the served generator's jobs, scaled down: sides 64..192, 200..600 steps, 2000 requests/s
    reqs = wl.serve_poisson(n_requests=n, rate_hz=2000.0, seed=8, side_max=192, steps_range=(200, 600), K=K)
    return reqs


def alone(job, blob):
    b = B.Batch(wl.F16_OFFSET, wl.MLP_BF16, K,
                B.pl_batch_overhead_bytes(2) + B.pl_batch_job_bytes(B.job_params(job)) + (1 << 20), max_jobs=2)
    b.set_weights(blob)
    jid = b.submit(job)
    assert jid is not None
    res = []
    while not res:
        b.advance(1)
        res = b.poll()
    b.close()
    return res[0]


def test_continuous_batching_results_match_jobs_alone():
    reqs = requests()
    blob = reqs[0].job.weights()
    per_job = max(B.pl_batch_job_bytes(B.job_params(r.job)) for r in reqs)
    budget = B.pl_batch_overhead_bytes(64) + 4 * per_job          # room for about four jobs
    srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, K, budget, blob, max_jobs=64)
    out = srv.run(reqs, max_wall_s=120.0)
    srv.close()
    assert out["jobs_done"] == len(reqs) and out["statuses"] == {0: len(reqs)}
    assert out["p50_latency_s"] is not None and out["p99_latency_s"] >= out["p50_latency_s"]
    res = sorted(out["results"], key=lambda r: r["request"])
    # memory was the limit: some request waited for a retirement
    assert max(r["admitted_s"] - reqs[r["request"]].arrival_s for r in res) > 0.0
    # continuous batching: a job admitted while another was still on the device
    overlap = any(a["admitted_interval"] > b["admitted_interval"] and a["admitted_interval"] < b["done_interval"]
                  for a in res for b in res)
    assert overlap
    for r in res:
        job = reqs[r["request"]].job
        ref = alone(job, blob)
        assert r["steps"] == ref["steps"] == -(-job.steps // K) * K
        assert r["status"] == ref["status"] == 0
        for k, v in ref["metrics"].items():   # (the Laplace fields are NaN for several droplets)
            w = r["metrics"][k]
            assert w == v or (np.isnan(w) and np.isnan(v)), (r["request"], k, w, v)

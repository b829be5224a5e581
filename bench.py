#!/usr/bin/env python
"""Throughput benchmark of the coupled PINN-LBM droplet hot path on GB300.

Metric: MLUPS (million lattice-cell updates per second) and the HBM-roofline
fraction of the fused collide-stream kernel; batched FP16-offset storage against
plain per-lattice FP32 storage; p50/p99 job latency of a served request stream.

One bench step = one coupling interval (arXiv 2504.10539 Sec. II-C) of the batched
workload: 256 independent periodic droplet lattices (side U{64..1024}, G U[-6,-5],
tau over the stable part of U[0.6,1.2], one centred droplet R U[0.1,0.35] side),
FP16-offset populations, FP32 arithmetic, BF16 tcgen05 network: K = 100 time steps
of every lattice, one interface correction (network inference on every cell +
projection + apply) and the metrics of every lattice, as one replayed CUDA graph.
The populations (2 x ~1.8 GB) exceed the 129 MB L2, so no flush is needed.

Also reported: the same 256 lattices run one by one with FP32 storage through the
single-lattice API ("fp32_plain"); a served Poisson request stream (continuous
batching, p50/p99 latency, offered vs served MLUPS); the single 4096x4096 droplet
field with FP16 and FP32 storage (step-kernel HBM fractions); the FP64 CPU oracle on
a bounded sample (cpu_baseline).  --impl reference times that oracle alone.
Multi-GPU (torchrun): every rank runs an independent replica of the same batch (weak
scaling, no collective on the data path).
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {0: 144, 1: 72, 2: 40}   # read + write of 9 populations (8 / 4 / 2 bytes); FP16-offset also its FP16 reference density
STORAGE_NAME = {0: "f64", 1: "f32", 2: "f16_offset"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lattices", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--serve-light-requests", type=int, default=60)
    ap.add_argument("--serve-light-rate", type=float, default=3.0)
    ap.add_argument("--field-side", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-field", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--train-side", type=int, default=512)
    ap.add_argument("--train-epochs", type=int, default=300)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def dist_max(dist, v, device):
    """Maximum of v over the ranks of the process group (v itself without one)."""
    import torch
    if dist is None:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(updates_per_rank, t_ms_max, world):
    """Whole-job throughput: the cell updates all ranks processed over the slowest rank's time."""
    return updates_per_rank * world / (t_ms_max / 1e3) / 1e6


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_index), "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_peaks_bf16():
    """Dense BF16 tensor peak (burst) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def step_kernel_hash():
    """Source hash of the step kernel (what the recorded DRAM traffic depends on)."""
    from paper_2504_10539_gb300 import build as PB
    return PB.source_hash(("pl_step.cu", "pl_device.cuh", "pl_kernels.h"))


def library_hash():
    """Source hash of the whole library (what the recorded accuracy depends on)."""
    from paper_2504_10539_gb300 import build as PB
    return PB.source_hash()


def profiled_traffic(key, units):
    """DRAM bytes of one step-kernel launch scaled from the committed ncu summary (taken on a
    smaller case; traffic grows with the cells updated), if it was taken on the current
    kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(key)
    if not e or e.get("kernel_sha1") != step_kernel_hash():
        return None
    return e["dram_bytes_per_cell_update"] * units


def oracle_interval(job, blob):
    """One coupling interval of `job` on the FP64 oracle: returns (cell updates, seconds)."""
    import oracle as O
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    M0 = O.mass(f)
    t0 = time.perf_counter()
    O.step(f, job.K, job.G, job.tau, job.rho0)
    O.correct(f, blob, job.beta_rho, job.beta_u, M0, O.MLP_F64)
    O.metrics_rho(O.density(f))
    return job.cells * job.K, time.perf_counter() - t0


def cpu_sample(jobs, budget_s):
    """The oracle on the batch's lattices, smallest first, one interval each, until budget_s."""
    import oracle as O
    O.set_num_threads(os.cpu_count() or 1)
    blob = jobs[0].weights()
    upd = secs = 0.0
    done = []
    for job in sorted(jobs, key=lambda j: j.cells):
        u, s = oracle_interval(job, blob)
        upd += u
        secs += s
        done.append("%dx%d" % (job.nx, job.ny))
        if secs > budget_s:
            break
    return upd, secs, done, O.num_threads()


def accuracy_record():
    """The full-length accuracy results (rho rel L-inf, W, mass drift against the FP64 oracle)
    as recorded by tests/test_gpu_accuracy.py on a GB300 (profiles/accuracy_full_length.json),
    marked stale if the library's source changed since."""
    p = os.path.join(ROOT, "profiles", "accuracy_full_length.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    rec["stale"] = rec.get("source_sha1") != library_hash()
    return rec


def oracle_run_rate(job, steps, threads):
    """MLUPS of the FP64 oracle on `steps` steps of `job` (with its corrections) on `threads`
    host threads: a bounded sample of the configuration, extrapolated per cell update."""
    import oracle as O
    O.set_num_threads(threads)
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    M0 = O.mass(f)
    mode = O.MLP_F64 if job.mlp == 0 else O.MLP_BF16
    t0 = time.perf_counter()
    O.run(f, steps, job.G, job.tau, K=job.K, blob=job.weights() if job.K else None, mode=mode,
          beta_rho=job.beta_rho, beta_u=job.beta_u, M0=M0)
    dt = time.perf_counter() - t0
    return job.cells * steps / dt / 1e6, dt


CONFIG_CASES = ("C1_single_64_fp64", "C2_single_512_fp32", "C3_field_4096_fp16", "C3_field_4096_fp32")


def config_jobs(wl):
    return {"C1_single_64_fp64": wl.single_64(), "C2_single_512_fp32": wl.single_512(),
            "C3_field_4096_fp16": wl.field_4096(storage=wl.F16_OFFSET),
            "C3_field_4096_fp32": wl.field_4096(storage=wl.F32)}


def config_runs(B, wl, torch):
    """Configurations 1-3 as configured, on the GPU: one run each through the single-lattice
    API (the first interval, which captures the graph, untimed), CUDA events on the lattice's
    stream."""
    out = {}
    jobs = config_jobs(wl)
    for name in CONFIG_CASES:
        job = jobs[name]
        lat = B.Lattice.from_workload(job)
        lat.run(job.K, job.K)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = job.steps - job.K
        e0.record(lat.stream)
        lat.run(steps, job.K)
        e1.record(lat.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        m = lat.metrics()
        lat.close()
        del lat
        torch.cuda.empty_cache()
        out[name] = {"workload": "%dx%d %s, %d steps, correction every %d (%s network)"
                                 % (job.nx, job.ny, STORAGE_NAME[job.storage], job.steps, job.K,
                                    {0: "FP64", 1: "FP32", 2: "BF16 tcgen05"}[job.mlp]),
                     "gpu_mlups": job.cells * steps / (ms / 1e3) / 1e6, "gpu_ms": ms, "status": m["status"]}
        if name.startswith("C3"):
            # the configured field breaks down in the FP64 oracle as well (recorded by
            # tests/golden/make_field_4096_stability.py): a non-physical final status is the
            # method's at this tau, not the storage's
            gold = os.path.join(ROOT, "tests", "golden", "field_4096_stability.json")
            if os.path.exists(gold):
                out[name]["oracle_plain_lbm_nonphysical_at_step"] = json.load(open(gold))["first_nonphysical_step"]
    return out


def config_oracle_rates(wl):
    """The FP64 oracle on a bounded sample of each of configurations 1-3, on one host thread and
    on all of them (per-cell-update rates extrapolated from the sample; the 4096^2 field is
    sampled on a 512^2 crop of its droplet density)."""
    jobs = config_jobs(wl)
    out = {}
    for name in CONFIG_CASES:
        if name == "C3_field_4096_fp32":            # the same FP64 computation as the FP16 case
            out[name] = out["C3_field_4096_fp16"]
            continue
        job, n = jobs[name], 100
        if name.startswith("C1"):
            n = 200
        if name.startswith("C3"):
            job = wl.field_4096(storage=job.storage, side=512, n_drop=6)
        r1, t1 = oracle_run_rate(job, n, 1)
        rn, tn = oracle_run_rate(job, n, os.cpu_count() or 1)
        out[name] = {"oracle_1_thread_mlups": r1, "oracle_all_threads_mlups": rn, "threads": os.cpu_count(),
                     "sample": "%dx%d, %d steps with its corrections (%.1f s on one thread, %.1f s on all), "
                               "MLUPS extrapolated per cell update" % (job.nx, job.ny, n, t1, tn)}
    return out


def batch_config(n_lattices, cells, K, world):
    """The workload keys both arms report (the GPU arm adds its launch configuration)."""
    return {"workload": "batch_%d" % n_lattices, "lattices": n_lattices, "cells": cells,
            "storage": "f16_offset", "network": "bf16-tcgen05", "K": K,
            "step": "one coupling interval: K lattice steps + correction + metrics of every lattice "
                    "(one CUDA graph replay)",
            "l2": "inputs larger than L2 (2 x %.2f GB populations)" % (cells * 20 / 1e9),
            "parallelism": "replicas x%d" % world}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2504_10539_gb300 import workloads as wl
    import oracle as O
    O.set_num_threads(os.cpu_count() or 1)
    jobs = sorted(wl.batch_256(n=args.lattices, seed=4), key=lambda j: j.cells)
    blob = jobs[0].weights()
    for k in range(min(args.warmup, 1)):
        oracle_interval(jobs[k % len(jobs)], blob)
    upd = secs = 0.0
    for k in range(args.steps):   # each step: one interval of one lattice, smallest lattices in turn
        u, s = oracle_interval(jobs[k % 8], blob)
        upd += u
        secs += s
    mlups = upd / secs / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(batch_config(args.lattices, sum(j.cells for j in jobs), 100, 1),
                       sample="FP64 CPU oracle: each step one coupling interval of one of the 8 smallest "
                              "lattices in turn"),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
                         "sample": "one coupling interval (K=100 steps + FP64 network correction + metrics) per "
                                   "step on the 8 smallest lattices of the batch in turn"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GB300 arm

# Training: algorithmic FLOPs per sample and epoch.  Three rows per sample (value and the two
# input tangents), each through the forward pass (33,088 multiply-adds), the reverse pass to
# the layer inputs (32,960: none into the 2 coordinates) and the weight gradient (33,088).
TRAIN_FLOP_PER_SAMPLE = 2 * 3 * (33088 + 32960 + 33088)
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz (maximum SM clock).
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def train_measurement(args, B, wl, torch, mode=0, cpu=True):
    """Sec. II-C step 2 at the paper's settings (lr 3e-4, 300 epochs per coupling round) on the
    single-droplet lattice of side --train-side (FP32 storage): epochs timed with CUDA events on
    the lattice's stream, then one full coupling round (K = 100 steps, training, correction).
    mode: PL_TRAIN_SIMT (FP32 CUDA cores) or PL_TRAIN_TC (BF16 tcgen05 layers 2-4 and gradients)."""
    side, E, K = args.train_side, args.train_epochs, 100
    job = wl.Lattice(side, side, storage=wl.F32, droplets=[(side / 2, side / 2, side * 80.0 / 512)], seed=2,
                     K=K, mlp=wl.MLP_BF16, weight_seed=12)
    lat = B.Lattice.from_workload(job)
    lat.step(K)
    tr = B.Trainer(lat, max_epochs=E, mode=mode)
    tr.train(min(3, E))                                     # warm-up (kernel set-up, first touch)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(lat.stream)
    tr.train(E)
    ev[1].record(lat.stream)
    ev[1].synchronize()
    hist = tr.losses(E)
    ev[2].record(lat.stream)
    tr.run(K, K, E)                                         # one coupling round: steps, training, correction
    ev[3].record(lat.stream)
    ev[3].synchronize()
    ms_epoch = ev[0].elapsed_time(ev[1]) / E
    round_ms = ev[2].elapsed_time(ev[3])
    tflops = job.cells * TRAIN_FLOP_PER_SAMPLE / (ms_epoch / 1e3) / 1e12
    m = lat.metrics()
    if mode == B.PL_TRAIN_TC:
        peak, kind = measured_peaks_bf16()
        roof = {"bound": "tensor", "kernel": "k_train_grad_tc + k_train_update<float>", "achieved": tflops,
                "peak": peak, "peak_kind": kind, "unit": "TFLOP/s", "frac": tflops / peak,
                "flop_per_sample": TRAIN_FLOP_PER_SAMPLE}
        arith = "BF16 tcgen05 layers 2-4 and the gradient sums, FP32 elsewhere"
    else:
        roof = {"bound": "alu", "kernel": "k_train_grad<float> + k_train_update<float>", "achieved": tflops,
                "peak": FP32_ALU_PEAK_TFLOPS, "peak_kind": "derived (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)",
                "unit": "TFLOP/s", "frac": tflops / FP32_ALU_PEAK_TFLOPS, "flop_per_sample": TRAIN_FLOP_PER_SAMPLE}
        arith = "FP32 training"
    out = {"workload": "%dx%d single droplet (R=%g), FP32 storage, %s, %d epochs per round, lr 3e-4"
                       % (side, side, side * 80.0 / 512, arith, E),
           "ms_per_epoch": ms_epoch, "samples_per_s": job.cells / (ms_epoch / 1e3),
           "roofline": roof,
           "round_ms": round_ms, "training_share_of_round": E * ms_epoch / round_ms,
           "loss_first_last": [hist[0, 0], hist[-1, 0]], "status_after_round": m["status"]}
    tr.close()
    lat.close()
    torch.cuda.empty_cache()
    if cpu and not args.no_cpu:
        import numpy as np
        import oracle as O
        import oracle.train as OT
        n = 128
        f = O.init_equilibrium(O.init_rho(n, n, [(n / 2, n / 2, n * 80.0 / 512)], 2.0, 0.15, 2.0, 0.01, 2))
        t0 = time.perf_counter()
        OT.train(job.weights(), f, 3, job.G)
        dt = (time.perf_counter() - t0) / 3
        out["cpu_baseline"] = {"value": n * n / dt, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "FP64 numpy training oracle, 3 epochs on a 128x128 lattice, %.2f s per epoch"
                                         % dt}
    return out


def run_gb300(args):
    import numpy as np
    import torch
    from paper_2504_10539_gb300 import binding as B
    from paper_2504_10539_gb300 import serve as S
    from paper_2504_10539_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return dist_max(dist, v, "cuda")

    peak, peak_kind = measured_peaks()
    gpu_index = local
    if "CUDA_VISIBLE_DEVICES" in os.environ:
        gpu_index = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])

    # --------------------------------------------------------------- batched FP16 (headline)
    K = 100
    n_e2e = 0 if args.no_e2e else min(args.steps, 5)
    n_int = args.warmup + args.steps + n_e2e + 2     # no job retires before the last timed interval
    # every rank runs the same batch (replicas: the per-GPU work is fixed as N grows, so the
    # updates of all ranks are the per-rank updates times N)
    jobs = wl.batch_256(n=args.lattices, seed=4, steps=n_int * K, K=K)
    blob = np.ascontiguousarray(jobs[0].weights())
    cells = sum(j.cells for j in jobs)
    budget = B.pl_batch_overhead_bytes(len(jobs) + 1) + sum(B.pl_batch_job_bytes(B.job_params(j)) for j in jobs)
    bt = B.Batch(wl.F16_OFFSET, wl.MLP_BF16, K, budget + (64 << 20), max_jobs=len(jobs) + 1)
    bt.set_weights(blob)
    for j in jobs:
        assert bt.submit(j) is not None
    rows_per_chunk = bt.autotune()
    for _ in range(args.warmup):
        bt.advance(1)
    B.pl_batch_interval_times(bt.h)
    clocks = ClockSampler(gpu_index)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.start()
    l0 = B.pl_kernel_launches()
    e0.record(bt.stream)
    step_ms, int_ms = [], []
    for _ in range(args.steps):
        bt.advance(1)
        s_ms, i_ms = B.pl_batch_interval_times(bt.h)   # events recorded inside the replayed interval
        step_ms.append(s_ms)
        int_ms.append(i_ms)
    e1.record(bt.stream)
    e1.synchronize()
    launches = B.pl_kernel_launches() - l0
    clk = clocks.stop()
    barrier()
    t_ms = max_over_ranks(e0.elapsed_time(e1))
    value = aggregate_mlups(cells * K * args.steps, t_ms, world)
    step_launch_ms = statistics.mean(step_ms) / K
    achieved = cells * BYTES_PER_UPDATE[wl.F16_OFFSET] / (step_launch_ms / 1e3) / 1e9
    live = B.pl_batch_metrics(bt.h)
    statuses = sorted({r["status"] for r in live})
    drift = max(abs(r["metrics"]["mass"] - r["metrics"]["mass0"]) / r["metrics"]["mass0"] for r in live)

    # end to end through the C ABI with host buffers: the weights uploaded from host memory
    # each interval (the paper retrains per coupling round) and every job's metric record read
    e2e = None
    if not args.no_e2e:
        rec_bytes = ctypes.sizeof(B.pl_job_result) * len(jobs)
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            B.pl_batch_set_mlp_weights(bt.h, blob)
            B.pl_batch_advance(bt.h, 1)
            B.pl_batch_metrics(bt.h)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        assert bt.info()["active"] == len(jobs), "a job retired inside the end-to-end region"
        e2e = {"value": cells * K * n_e2e * world / t_e2e / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(blob.nbytes), "d2h_bytes_per_step": int(rec_bytes)}
    bt.close()
    del bt
    torch.cuda.empty_cache()

    # --------------------------------------------------------------- plain per-lattice FP32
    fp32 = None
    if not args.no_fp32 and world == 1:     # a per-GPU comparison: one GPU only
        lats = []
        t_plain = 0.0
        n_plain = 2
        for j in jobs:
            j32 = wl.Lattice(**{**j.__dict__, "storage": wl.F32, "mlp": wl.MLP_BF16})
            lat = B.Lattice(B.job_params(j32))
            lat.init_droplets(j32.droplets, j32.rho_in, j32.rho_out, j32.width, j32.noise_amp, j32.seed)
            lat.set_weights(blob)
            lat.run(K, K)                              # warm-up interval (graph capture)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(lat.stream)
            lat.run(n_plain * K, K)
            ev1.record(lat.stream)
            ev1.synchronize()
            t_plain += ev0.elapsed_time(ev1)
            lat.close()
            del lat
        torch.cuda.empty_cache()
        v32 = cells * K * n_plain / (t_plain / 1e3) / 1e6
        fp32 = {"value": v32, "unit": "MLUPS", "form": "each lattice alone, single-lattice API, FP32 storage, "
                                                       "BF16 network, graph per interval",
                "speedup_batched_f16_over_plain_f32": value / v32}

    # --------------------------------------------------------------- served request streams
    serving = None
    if not args.no_serve and rank == 0 and world == 1:
        serving = {}
        legs = [("saturated", args.serve_requests, 200.0), ("sub_capacity", args.serve_light_requests,
                                                            args.serve_light_rate)]
        for leg, n_req, rate in legs:
            reqs = wl.serve_poisson(n_requests=n_req, rate_hz=rate, seed=5)
            srv = S.Server(wl.F16_OFFSET, wl.MLP_BF16, K, 150 * (1 << 30), reqs[0].job.weights(), max_jobs=1024)
            out = srv.run(reqs, max_wall_s=300.0)
            srv.close()
            torch.cuda.empty_cache()
            rec = {k: out[k] for k in ("jobs_done", "jobs_submitted", "jobs_rejected", "p50_latency_s",
                                       "p99_latency_s", "p50_queue_wait_s", "p99_queue_wait_s", "served_mlups",
                                       "offered_mlups", "elapsed_s", "intervals", "peak_active_jobs")}
            rec["statuses"] = {str(k): v for k, v in out["statuses"].items()}
            rec["workload"] = ("Poisson %g req/s, side U{64..2048 step 32}, 1-8 droplets, G U[-6,-5], "
                               "steps U[1000,20000] rounded up to K=100, 150 GB budget, %d requests" % (rate, n_req))
            serving[leg] = rec

    # --------------------------------------------------------------- single 4096^2 field
    field = None
    if not args.no_field and world == 1:
        field = {}
        for st in (wl.F16_OFFSET, wl.F32):
            job = wl.field_4096(storage=st, side=args.field_side)
            job.mlp = wl.MLP_BF16
            lat = B.Lattice.from_workload(job)
            lat.step(K)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            for a, b in ev:
                a.record(lat.stream)
                lat.step(K)
                b.record(lat.stream)
                lat.correct()
            m = lat.metrics()
            ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / K
            gbs = job.cells * BYTES_PER_UPDATE[st] / (ms / 1e3) / 1e9
            field[STORAGE_NAME[st]] = {"step_kernel_ms": ms, "GBps": gbs, "frac": gbs / peak,
                                       "mlups_steps_only": job.cells / (ms / 1e3) / 1e6,
                                       "mass_drift_post_correction": abs(m["mass"] - m["mass0"]) / m["mass0"],
                                       "traffic": profiled_traffic("%s_field" % STORAGE_NAME[st], job.cells)}
            lat.close()
            del lat
            torch.cuda.empty_cache()
        # the correction's share of a coupling interval, the full correction against the interface
        # band of mask_eps = 0.01 (the network evaluated on the band only)
        band = {}
        for eps in (0.0, 0.01):
            job = wl.field_4096(storage=wl.F16_OFFSET, side=args.field_side)
            job.mask_eps = eps
            lat = B.Lattice.from_workload(job)
            lat.step(K)
            lat.correct()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(lat.stream)
            lat.step(K)
            ev[1].record(lat.stream)
            lat.correct()
            ev[2].record(lat.stream)
            ev[2].synchronize()
            steps_ms, corr_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
            m = lat.metrics()
            band["eps_%g" % eps] = {"steps_ms": steps_ms, "correction_ms": corr_ms,
                                    "correction_share_of_interval": corr_ms / (steps_ms + corr_ms),
                                    "status": m["status"]}
            lat.close()
            del lat
            torch.cuda.empty_cache()
        field["correction_band"] = band

    # --------------------------------------------------------------- network training (Eqs. 3-8)
    training = training_tc = None
    if not args.no_train and rank == 0 and world == 1:
        training = train_measurement(args, B, wl, torch, B.PL_TRAIN_SIMT)
        training_tc = train_measurement(args, B, wl, torch, B.PL_TRAIN_TC, cpu=False)

    # --------------------------------------------------------------- configurations 1-3
    configs = None
    if not args.no_configs and rank == 0 and world == 1:
        configs = config_runs(B, wl, torch)

    # --------------------------------------------------------------- CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        upd, secs, done, cores = cpu_sample(jobs, 12.0)
        cpu = {"value": upd / secs / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle, one coupling interval (K=100 steps + FP64 network correction + metrics) of "
                         "the %d smallest lattices of the batch (%s), %.1f s" % (len(done), ", ".join(done), secs)}
        if not args.no_configs:
            cpu["per_config"] = config_oracle_rates(wl)

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(batch_config(len(jobs), cells, K, world), rows_per_chunk=rows_per_chunk),
            "roofline": {"bound": "hbm", "kernel": "k_step<f16_offset> (batched)", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profiled_traffic("f16_offset_batch", cells),
                         "algorithmic_bytes_per_launch": cells * BYTES_PER_UPDATE[wl.F16_OFFSET],
                         "step_kernel_ms": step_launch_ms,
                         "interval_ms_mean": statistics.mean(int_ms)},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons", [])},
            "fp32_plain": fp32,
            "serving": serving,
            "field_4096": field,
            "training": training,
            "training_tc": training_tc,
            "configs": configs,
            "accuracy": accuracy_record(),
            "cpu_baseline": cpu,
            "batch_checks": {"statuses": statuses, "max_mass_drift_post_correction": drift},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gb300(a)

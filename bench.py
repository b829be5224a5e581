#!/usr/bin/env python
"""Throughput benchmark of the coupled PINN-LBM droplet hot path on GB300.

Metric: MLUPS (million lattice-cell updates per second) and the HBM-roofline
fraction of the fused collide-stream kernel, FP16-offset storage against plain
FP32 storage.

One bench step = one coupling interval of the method (arXiv 2504.10539 Sec. II-C):
K = 100 time steps of Eq. 1, one interface correction (network inference on
every cell + projection + apply) and the interface metrics (Eqs. 9-16), read
back to the host.  Workload: the 4096x4096 periodic coalescence field
(400 droplets, radii U[8,40], tau = 0.8, G = -5.5), FP16-offset populations
with FP32 arithmetic and the BF16 tensor-core network (FP32 network until the
tensor-core kernel is in), synthetic seeded input.  Both population buffers
(2 x 302 MB) exceed the 129 MB L2, so no L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle (test infrastructure) on the host
cores on a bounded crop of the same workload.
Multi-GPU (torchrun): every rank runs an independent replica of the field
(weak scaling, no collective on the data path).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {0: 144, 1: 72, 2: 36}   # read + write of 9 populations (8 / 4 / 2 bytes)
STORAGE_NAME = {0: "f64", 1: "f32", 2: "f16_offset"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--mlp", default="auto", choices=["auto", "bf16", "f32"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--storage", default="f16", choices=["f16", "f32"],
                    help="storage of the timed workload (profiling aid; the headline is f16)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
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
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def step_kernel_hash():
    h = hashlib.sha1()
    for f in ("pl_step.cu", "pl_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2504_10539_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(storage, side):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get("%s_%d" % (STORAGE_NAME[storage], side))
    if not e or e.get("kernel_sha1") != step_kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


def cpu_sample_workload(side):
    from paper_2504_10539_gb300 import workloads as wl
    # same droplet density and radius distribution as the full field
    n_drop = max(1, round(400 * (side / 4096.0) ** 2))
    return wl.field_4096(storage=wl.F16_OFFSET, side=side, n_drop=n_drop)


def time_oracle(job, steps, budget_s=None):
    """Run the FP64 oracle on `job` for `steps` bench steps (K LBM steps + correction +
    metrics each) or until budget_s elapsed; returns (updates, seconds, steps_done)."""
    import oracle as O
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    M0 = O.mass(f)
    blob = job.weights()
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        O.step(f, job.K, job.G, job.tau, job.rho0)
        O.correct(f, blob, job.beta_rho, job.beta_u, M0, O.MLP_F64)
        O.metrics_rho(O.density(f))
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return job.cells * job.K * done, dt, done


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    job = cpu_sample_workload(512)
    O.set_num_threads(os.cpu_count() or 1)
    # each bench step is one coupling interval on the 512x512 crop
    for _ in range(args.warmup if args.warmup < 1 else 1):
        time_oracle(job, 1)
    upd, dt, done = time_oracle(job, args.steps)
    mlups = upd / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": done, "warmup": args.warmup, "ms_per_step": dt * 1e3 / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "field_%d crop 512x512 (FP64 CPU oracle)" % args.side, "K": job.K,
                   "droplets": len(job.droplets)},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
                         "sample": "512x512 crop of the droplet field (%d droplets), %d coupling intervals of "
                                   "K=%d steps + FP64 network correction + metrics" % (len(job.droplets), done, job.K)},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GB300 arm

def run_gb300(args):
    import numpy as np
    import torch
    from paper_2504_10539_gb300 import binding as B
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
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    mlp = {"auto": wl.MLP_BF16, "bf16": wl.MLP_BF16, "f32": wl.MLP_F32}[args.mlp]

    def build(storage):
        job = wl.field_4096(storage=storage, seed=3 + rank, side=args.side)
        job.mlp = mlp
        return job, B.Lattice.from_workload(job)

    def time_workload(storage, steps, warmup, with_clocks):
        job, lat = build(storage)
        s = lat.stream
        K = job.K
        for _ in range(warmup):
            lat.step(K)
            lat.correct()
            lat.metrics()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local])
                              if "CUDA_VISIBLE_DEVICES" in os.environ else local) if with_clocks else None
        barrier()
        if clocks:
            clocks.start()
        l0 = B.pl_kernel_launches()
        e0.record(s)
        for k in range(steps):
            ev[k][0].record(s)
            lat.step(K)                  # K fused collide-stream launches
            ev[k][1].record(s)
            lat.correct()                # network + projection + apply
            m = lat.metrics()            # Eqs. 9-16, FP64 record to the host
        e1.record(s)
        e1.synchronize()
        launches = B.pl_kernel_launches() - l0
        clk = clocks.stop() if clocks else None
        barrier()
        t_ms = max_over_ranks(e0.elapsed_time(e1))
        step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / K  # per step-kernel launch
        assert m["status"] == 0, m
        res = {"job": job, "t_ms": t_ms, "step_kernel_ms": step_ms, "launches": launches, "clocks": clk,
               "metrics": m}
        return res, lat

    storage = wl.F16_OFFSET if args.storage == "f16" else wl.F32
    def measure_drift(lat, K):
        """Relative mass drift |M - M0| / M0 after the timed region: one more interval,
        read before and after its correction (whose projection targets M0)."""
        lat.step(K)
        pre = lat.metrics()
        lat.correct()
        post = lat.metrics()
        M0 = post["mass0"]
        return {"pre_correction": abs(pre["mass"] - M0) / M0, "post_correction": abs(post["mass"] - M0) / M0,
                "after_steps": post["step"]}

    main, lat = time_workload(storage, args.steps, args.warmup, True)
    drift = measure_drift(lat, main["job"].K)
    job = main["job"]
    K = job.K
    cells = job.cells
    updates = cells * K * args.steps * world
    value = updates / (main["t_ms"] / 1e3) / 1e6
    peak, peak_kind = measured_peaks()
    achieved = cells * BYTES_PER_UPDATE[storage] / (main["step_kernel_ms"] / 1e3) / 1e9
    traffic = profiled_traffic(storage, args.side)

    # end to end through the C ABI with host buffers: new network weights uploaded each
    # interval (the paper retrains per coupling round), metrics record read back
    e2e = None
    if not args.no_e2e:
        blob = np.ascontiguousarray(job.weights())
        rec = B.pl_metric_record()
        n_e2e = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            B.pl_set_mlp_weights(lat.h, blob)
            B.pl_step(lat.h, K)
            B.pl_apply_correction(lat.h)
            B.pl_metrics(lat.h)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": cells * K * n_e2e * world / t_e2e / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(blob.nbytes), "d2h_bytes_per_step": ctypes.sizeof(rec)}
    lat.close()
    del lat
    torch.cuda.empty_cache()

    fp32 = None
    if not args.no_fp32:
        r32, lat32 = time_workload(wl.F32, max(3, args.steps // 2), 1, False)
        drift32 = measure_drift(lat32, K)
        lat32.close()
        del lat32
        torch.cuda.empty_cache()
        v32 = cells * K * max(3, args.steps // 2) * world / (r32["t_ms"] / 1e3) / 1e6
        a32 = cells * BYTES_PER_UPDATE[wl.F32] / (r32["step_kernel_ms"] / 1e3) / 1e9
        fp32 = {"value": v32, "unit": "MLUPS", "step_kernel_GBps": a32, "frac": a32 / peak,
                "speedup_f16_over_f32": value / v32, "mass_drift": drift32}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        O.set_num_threads(os.cpu_count() or 1)
        sjob = cpu_sample_workload(512)
        upd, dt, done = time_oracle(sjob, 20, budget_s=12.0)
        cpu = {"value": upd / dt / 1e6, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
               "sample": "512x512 crop of the field (%d droplets), %d coupling intervals of K=%d steps + FP64 "
                         "network correction + metrics, %.1f s" % (len(sjob.droplets), done, sjob.K, dt)}

    if rank == 0:
        clk = main["clocks"] or {}
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["t_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "field_%d" % args.side, "lattice": "%dx%d periodic D2Q9" % (args.side, args.side),
                       "storage": STORAGE_NAME[storage], "network": {wl.MLP_BF16: "bf16-tcgen05",
                                                                     wl.MLP_F32: "f32-simt"}[mlp],
                       "droplets": len(job.droplets), "tau": job.tau, "G": job.G, "K": K,
                       "step": "K lattice steps + correction + metrics",
                       "l2": "inputs larger than L2 (2 x %.0f MB populations)" % (cells * 18 / 1e6),
                       "parallelism": "replicas x%d" % world},
            "roofline": {"bound": "hbm", "kernel": "k_step<%s>" % STORAGE_NAME[storage], "achieved": achieved,
                         "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": cells * BYTES_PER_UPDATE[storage],
                         "step_kernel_ms": main["step_kernel_ms"]},
            "e2e": e2e,
            "gpu_launches": main["launches"],
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons", [])},
            "fp32_plain": fp32,
            "cpu_baseline": cpu,
            "final_metrics": {k: main["metrics"][k] for k in ("mass", "mass0", "W", "G_max", "W_eff", "E_int")},
            "mass_drift": drift,
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

"""Writes oracle_conditioning.json: how far the FP64 oracle's own coupled runs move when their
initial populations are rounded once to FP32.

Test infrastructure: it calls only the oracle (and the seeded workload descriptions).  The
coupled runs of Sec. II-C on a coalescing field are dynamically sensitive: a perturbation at
FP32's last place grows with the run.  The number recorded here is the relative L-inf distance
(on rho) between the oracle's run from the exact initial state and its run from that state
rounded to FP32, at each checkpoint: the least error any implementation that stores its
populations in FP32 at any time can be expected to show at that length.  The GPU accuracy tests
use it where it exceeds the fixed bounds.

    python tests/golden/make_oracle_conditioning.py [threads]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2504_10539_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_conditioning.json")


def init(job):
    return O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                         job.noise_amp, job.seed))


def run(job, f, mode, checkpoints):
    M0 = O.mass(f)
    out, s = {}, 0
    for c in checkpoints:
        st = O.run(f, c - s, job.G, job.tau, K=job.K, blob=job.weights() if job.K else None, mode=mode,
                   beta_rho=job.beta_rho, beta_u=job.beta_u, M0=M0, step0=s)
        assert st == 0, (job.nx, c, st)
        s = c
        out[c] = O.density(f).copy()
    return out


def sensitivity(job, mode, checkpoints):
    f = init(job)
    a = run(job, f.copy(), mode, checkpoints)
    b = run(job, f.astype(np.float32).astype(np.float64), mode, checkpoints)
    return {str(c): float(np.abs(a[c] - b[c]).max() / np.abs(a[c]).max()) for c in checkpoints}


def c3_crop(mlp, K=100):
    job = wl.field_4096(storage=wl.F32, side=512, n_drop=400 * 512 * 512 // (4096 * 4096))
    job.mlp, job.K = mlp, K
    return job


def main():
    if len(sys.argv) > 1:
        O.set_num_threads(int(sys.argv[1]))
    res = {"perturbation": "initial populations rounded once to FP32 (round to nearest)",
           "measure": "relative L-inf distance on rho between the two oracle runs"}
    # the 512^2 window of the 4096^2 coalescence field (400 droplets per 4096^2, radii 8-40,
    # G -5.5, tau 0.8), correction every 100 steps with the FP64 network and without correction
    steps = [1000, 2000, 3000, 4000, 5000]
    res["C3_field_512_fp64net"] = sensitivity(c3_crop(wl.MLP_F32), O.MLP_F64, steps)
    res["C3_field_512_pure"] = sensitivity(c3_crop(wl.MLP_F32, K=0), O.MLP_F64, steps)
    # lattices of the 256-lattice batch through its 2000 steps (correction every 100 steps, the
    # BF16 network emulated in the oracle)
    jobs = wl.batch_256()
    res["C4_batch"] = {str(k): sensitivity(jobs[k], O.MLP_BF16, [2000])["2000"] for k in (12, 102)}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()

"""Writes oracle_conditioning.json: how far the FP64 oracle's own coupled runs move under FP32
rounding of their state.

Test infrastructure: it calls only the oracle (and the seeded workload descriptions).  Two
perturbations of the oracle's run, each measured as the relative L-inf distance on rho from the
unperturbed run at each checkpoint:
  - "once": the initial populations rounded to FP32 (round to nearest), then FP64 throughout;
  - "every_step": the populations rounded to FP32 after every step (FP64 arithmetic with FP32
    storage: the rounding any FP32-storage implementation applies, without the rounding of its
    arithmetic).
The runs of Sec. II-C damp a single perturbation, but one applied at every step can grow: the
"every_step" distance is the least error an FP32-storage run can be expected to show at that
length.  The GPU accuracy tests bound an FP32 run by ten times it where that exceeds the fixed
bound (FP32 arithmetic adds about ten roundings per population and step to the storage's one),
and treat a run whose "every_step" distance alone exceeds its storage's bound as beyond the
reach of that bound.

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


def run_rounded(job, f, mode, checkpoints):
    """The oracle's run with the populations rounded to FP32 after every step."""
    M0 = O.mass(f)
    blob = job.weights() if job.K else None
    out, s = {}, 0
    for c in checkpoints:
        while s < c:
            corr = job.K > 0 and (s + 1) % job.K == 0
            st = O.run(f, 1, job.G, job.tau, K=job.K if corr else 0, blob=blob if corr else None, mode=mode,
                       beta_rho=job.beta_rho, beta_u=job.beta_u, M0=M0, step0=s)
            assert st == 0, (job.nx, s, st)
            f[...] = f.astype(np.float32).astype(np.float64)
            s += 1
        out[c] = O.density(f).copy()
    return out


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def sensitivity(job, mode, checkpoints):
    f = init(job)
    a = run(job, f.copy(), mode, checkpoints)
    b = run(job, f.astype(np.float32).astype(np.float64), mode, checkpoints)
    e = run_rounded(job, f.copy(), mode, checkpoints)
    return {"once": {str(c): rel(b[c], a[c]) for c in checkpoints},
            "every_step": {str(c): rel(e[c], a[c]) for c in checkpoints}}


def c3_crop(mlp, K=100):
    job = wl.field_4096(storage=wl.F32, side=512, n_drop=400 * 512 * 512 // (4096 * 4096))
    job.mlp, job.K = mlp, K
    return job


def main():
    if len(sys.argv) > 1:
        O.set_num_threads(int(sys.argv[1]))
    res = {"perturbations": {"once": "initial populations rounded once to FP32 (round to nearest)",
                             "every_step": "populations rounded to FP32 after every step"},
           "measure": "relative L-inf distance on rho from the unperturbed oracle run"}
    # the 512^2 coalescence field of the accuracy tests (the 4096^2 field's droplet density, 400
    # per 4096^2, radii 8-40, G -5.5, tau 0.8), correction every 100 steps with the FP64 network
    steps = [1000, 2000, 3000, 4000, 5000]
    res["C3_field_512_fp64net"] = sensitivity(c3_crop(wl.MLP_F32), O.MLP_F64, steps)
    # lattices of the 256-lattice batch through its 2000 steps (correction every 100 steps, the
    # BF16 network emulated in the oracle)
    jobs = wl.batch_256()
    res["C4_batch"] = {str(k): sensitivity(jobs[k], O.MLP_BF16, [1000, 2000]) for k in (12, 102)}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()

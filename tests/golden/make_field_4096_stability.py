"""Writes field_4096_stability.json: the step at which the FP64 oracle's plain LBM (no
correction) of the 4096^2 coalescence field first holds a non-finite density.

Test infrastructure: it calls only the oracle (and the seeded workload description).  The
configured field (400 droplets, radii 8-40, G -5.5, tau 0.8, started at the coexistence
densities) is dynamically unstable at this tau: a vapour region is driven through zero density
and the state becomes non-finite.  The oracle runs in chunks of 100 steps and records, after
each chunk, the minimum density and whether every density is finite, up to the first chunk
that ends non-finite.  `tests/test_gpu_fullsize.py` checks that the GPU's FP32 run of the same
field turns non-physical in the same chunk.  About 3.6e10 cell updates: tens of minutes on a
multi-core host.

    python tests/golden/make_field_4096_stability.py [threads]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2504_10539_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "field_4096_stability.json")
CHUNK = 100


def main():
    if len(sys.argv) > 1:
        O.set_num_threads(int(sys.argv[1]))
    job = wl.field_4096(storage=wl.F32)
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    log, first_bad = [], None
    t0 = time.time()
    for s in range(CHUNK, job.steps + 1, CHUNK):
        O.run(f, CHUNK, job.G, job.tau, K=0)
        r = O.density(f)
        bad = ~np.isfinite(r) | (r <= 0.0)
        rec = {"step": s, "physical": not bool(bad.any()), "rho_min": float(np.nanmin(r)),
               "secs": round(time.time() - t0, 1)}
        if bad.any():
            ys, xs = np.nonzero(bad)
            rec["bad_cells"] = int(bad.sum())
            rec["bad_box"] = [int(xs.min()), int(xs.max()), int(ys.min()), int(ys.max())]
        log.append(rec)
        print(json.dumps(rec), flush=True)
        if bad.any():
            first_bad = s
            break
    res = {"workload": "4096^2 coalescence field, 400 droplets (radii 8-40), G -5.5, tau 0.8, plain LBM, FP64 oracle",
           "chunk_steps": CHUNK, "first_nonphysical_step": first_bad, "chunks": log}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()

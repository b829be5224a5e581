"""The paper's simulation protocol (arXiv 2504.10539 Sec. III-C) on one droplet lattice.

  1. initialisation: `init_steps` (500) pure LBM steps to form the droplet;
  2. coupling: `K` steps, then training with epochs[0] (300, Sec. III-B) epochs, then the
     interface correction;
  3. evolution: len(epochs) - 1 further rounds of K steps + training + correction, with the
     epoch counts epochs[1:] (the paper gives no values, only that they decrease; the default
     250, 200, 150, 100, 50 decreases linearly);
  4. comparison: a pure LBM copy of the lattice, taken after the initialisation, advances the
     same number of steps;
  5. evaluation: the interface metrics (Eqs. 9-15) of both lattices after every round, and of
     the initialisation every `record_every` steps (the series of Figs. 1 and 3).

The steps per round (K = 100) are this library's reading of the few LBM steps between
corrections that Sec. II-C calls for, as in the single-droplet workloads.  Every number comes
from the library's kernels (C ABI ``pl_step``, ``pl_train``, ``pl_apply_correction``,
``pl_metrics``); this module only orders the calls.
"""
from __future__ import annotations

import json
import sys
from typing import Dict, Sequence

from . import binding as B
from . import workloads as wl

METRICS = ("W", "G_max", "delta_rho", "W_eff", "E_int", "mass")
DEFAULT_EPOCHS = (300, 250, 200, 150, 100, 50)


def _pick(m):
    return {k: m[k] for k in METRICS}


def run(job: wl.Lattice, init_steps: int = 500, K: int = 100, epochs: Sequence[int] = DEFAULT_EPOCHS,
        record_every: int = 50, hyper: Dict = None) -> Dict:
    """Runs the protocol on `job` (its initial state, storage, physics and seeded weights).

    Returns {"init": [(step, metrics)], "pinn": [(step, epochs, metrics, losses)],
    "pure": [(step, metrics)]}; losses = (first, last) total loss of the round's training."""
    hyper = hyper or {}
    pinn = B.Lattice(B.job_params(job))
    pinn.init_droplets(job.droplets, job.rho_in, job.rho_out, job.width, job.noise_amp, job.seed)
    pinn.set_weights(job.weights())
    out = {"init": [(0, _pick(pinn.metrics()))], "pinn": [], "pure": []}
    done = 0
    while done < init_steps:
        n = min(record_every, init_steps - done)
        pinn.step(n)
        done += n
        out["init"].append((done, _pick(pinn.metrics())))
    # the pure-LBM arm starts from the same state
    pure = B.Lattice(B.job_params(job))
    f, step = pinn.state()
    pure.set_state(f, step)
    trainer = B.Trainer(pinn, max_epochs=max(epochs), **hyper)
    for e in epochs:
        pinn.step(K)
        trainer.train(e)
        h = trainer.losses(e)
        pinn.correct()
        pure.step(K)
        done += K
        out["pinn"].append((done, int(e), _pick(pinn.metrics()), (float(h[0, 0]), float(h[-1, 0]))))
        out["pure"].append((done, _pick(pure.metrics())))
    out["status"] = {"pinn": pinn.status(), "pure": pure.status()}
    trainer.close()
    pinn.close()
    pure.close()
    return out


if __name__ == "__main__":
    side = int(sys.argv[1]) if len(sys.argv) > 1 else 256
    job = wl.Lattice(side, side, storage=wl.F32, droplets=[(side / 2, side / 2, side / 6)], mlp=wl.MLP_BF16, K=100)
    print(json.dumps(run(job)))

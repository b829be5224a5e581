"""Parity at the benchmark's full sizes, in the launch configuration the benchmark times.

The oracle cannot run the full workloads in a test's time, so these checks sample:

* the 4096x4096 coalescence field: a seeded droplet field of the workload's structure (400
  droplets, the field's densities), stored exactly in the lattice's storage type, advanced one
  step on the GPU (FP16-offset and FP32 storage) and compared on windows against the oracle's
  step of the same window of the same state.  A cell's post-streaming value depends on
  populations at most two cells away (streaming from a neighbour whose force reads its
  neighbours' density), so the window interior at distance >= 3 from the window edge is exact
  even though the oracle treats the window as periodic.  Windows are placed at random,
  including across the periodic boundary.
* the 256-lattice batch: all 256 lattices in one table, one coupling interval of K = 1 step
  (step + correction + metrics: the same table kernels and grids the benchmark replays with
  K = 100); the smallest lattices are compared whole against the oracle's own initial state,
  step and correction; every lattice must end with status OK and its mass at M0.
* the 4096x4096 field as configured, plain LBM: it breaks down (a density through zero) in the
  same 100-step chunk and region as the FP64 oracle's run of it.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import seeded_states as S
from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

MARGIN = 3
WIN = 48


def window(f, x0, y0, n):
    """n x n window of f[9][ny][nx] starting at (x0, y0), periodic."""
    _, ny, nx = f.shape
    ys = (y0 + np.arange(n)) % ny
    xs = (x0 + np.arange(n)) % nx
    return f[:, ys][:, :, xs]


# absolute bounds: FP16-offset storage keeps each population as an offset from its source
# cell's rest equilibrium; after one step from rest those offsets are below 1/8 in magnitude,
# where the FP16 spacing is at most 2^-14 (a moving population within half of it, the rest
# population within one spacing of its own plus the moving ones' errors); FP32 storage: a few
# FP32 roundings of values near 1
@pytest.mark.parametrize("storage,tol", [(wl.F16_OFFSET, 2.0 ** -12), (wl.F32, 2e-6)])
def test_field_4096_one_step_sampled_windows(storage, tol):
    job = wl.field_4096(storage=storage)
    rho = S.droplet_field_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width, job.noise_amp, 17)
    f0 = S.stored(S.at_rest(rho), storage)
    del rho
    lat = B.Lattice(B.job_params(job))
    lat.set_state(f0, 0)
    lat.step(1)
    f1, step = lat.state()
    assert step == 1
    rng = np.random.default_rng(7)
    corners = [(0, 0), (job.nx - WIN // 2, job.ny - WIN // 2)] + [tuple(rng.integers(0, job.nx, 2)) for _ in range(6)]
    worst = 0.0
    for x0, y0 in corners:
        w0 = window(f0, x0, y0, WIN).copy()
        O.step(w0, 1, job.G, job.tau)
        w1 = window(f1, x0, y0, WIN)
        inner = (slice(None), slice(MARGIN, WIN - MARGIN), slice(MARGIN, WIN - MARGIN))
        err = np.abs(w1[inner] - w0[inner]).max()
        worst = max(worst, err)
    assert worst <= tol, worst


def test_batch_256_one_interval_sampled_lattices():
    K = 1
    jobs = wl.batch_256(steps=K, K=K)
    blob = jobs[0].weights()
    budget = B.pl_batch_overhead_bytes(len(jobs)) + sum(B.pl_batch_job_bytes(B.job_params(j)) for j in jobs) + (64 << 20)
    bt = B.Batch(wl.F16_OFFSET, wl.MLP_BF16, K, budget, max_jobs=len(jobs))
    bt.set_weights(blob)
    ids = [bt.submit(j, steps=4 * K) for j in jobs]
    assert all(i is not None for i in ids)
    order = sorted(range(len(jobs)), key=lambda k: jobs[k].cells)
    bt.advance(1)
    live = {r["id"]: r for r in B.pl_batch_metrics(bt.h)}
    assert len(live) == len(jobs)
    for k, jid in enumerate(ids):
        m = live[jid]["metrics"]
        assert live[jid]["status"] == 0, (k, live[jid])
        assert m["corrections"] == 1
        assert abs(m["mass"] - m["mass0"]) <= 1e-6 * m["mass0"], k
    for k in order[:6]:
        j = jobs[k]
        fo = O.init_equilibrium(O.init_rho(j.nx, j.ny, j.droplets, j.rho_in, j.rho_out, j.width, j.noise_amp,
                                           j.seed))
        M0 = O.mass(fo)
        O.step(fo, 1, j.G, j.tau)
        assert O.correct(fo, blob, j.beta_rho, j.beta_u, M0, O.MLP_BF16) == 0
        f1, step = bt.state(ids[k])
        assert step == K
        # FP16 offsets of the initial state, of the step and of the correction (each below
        # 2^-14 here), the network in BF16 on both sides (the oracle emulates its rounding)
        assert np.abs(f1 - fo).max() <= 1e-3, (k, j.nx, np.abs(f1 - fo).max())
    bt.close()


# ----------------------------------------------------------------------------- breakdown

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "field_4096_stability.json")


@pytest.mark.parametrize("storage", [wl.F32, wl.F16_OFFSET])
def test_field_4096_plain_lbm_breaks_down_where_the_oracle_does(storage):
    """The configured 4096^2 field is dynamically unstable at tau = 0.8: the FP64 oracle's plain
    LBM holds a non-finite density after the chunk recorded in tests/golden/ (written by
    make_field_4096_stability.py, which runs the oracle only).  The GPU run of the same field
    (as configured, full size, without correction) turns non-physical in the same chunk of 100
    steps, or one chunk either side, and its first non-physical cells lie in the region where
    the oracle's did (within 64 cells)."""
    gold = json.load(open(GOLD))
    s_bad = gold["first_nonphysical_step"]
    x0, x1, y0, y1 = gold["chunks"][-1]["bad_box"]
    chunk = gold["chunk_steps"]
    job = wl.field_4096(storage=storage)
    job.K = 0
    lat = B.Lattice.from_workload(job)
    first = None
    for s in range(chunk, s_bad + 2 * chunk + 1, chunk):
        lat.step(chunk)
        if lat.metrics()["status"] != 0:
            first = s
            break
    assert first is not None and abs(first - s_bad) <= chunk, (first, s_bad)
    r = lat.rho()
    lat.close()
    ys, xs = np.nonzero(~np.isfinite(r) | (r <= 0.0))
    assert len(xs) > 0
    near = (xs >= x0 - 64) & (xs <= x1 + 64) & (ys >= y0 - 64) & (ys <= y1 + 64)
    assert near.any(), (xs.min(), xs.max(), ys.min(), ys.max(), gold["chunks"][-1]["bad_box"])


# ----------------------------------------------------------------------------- largest planes

# 20736^2 cells: ten FP16 planes span 4.3e9 elements, past 32-bit element offsets, so the FP16
# step takes its element-by-element path with 64-bit offsets (the vector path's offsets are 32
# bits); FP32 storage of the same size always uses 64-bit offsets.  About 31 / 43 GB of device
# memory and 7 GB of host memory.
BIG = 20736


@pytest.mark.parametrize("storage,tol", [(wl.F16_OFFSET, 2e-4), (wl.F32, 1e-6)])
def test_planes_beyond_32_bit_element_offsets(storage, tol):
    """One step of a 20736^2 lattice from rest on a seeded random density field, compared on
    windows, including the last rows (the largest offsets) and across the periodic edges, with
    the oracle's step of the same window (interior at distance >= 3 exact, as above).  Bounds:
    FP32 a few FP32 roundings; FP16-offset the initial encoding (moving offsets up to ~11 in
    2^-10 units, whose FP16 spacing is 2^-7: 3.8e-6 per population, nine arriving per cell)."""
    assert 10 * BIG * BIG > 2 ** 32
    p = B.pl_params_default(BIG, BIG, storage=storage)
    rng = np.random.default_rng(5)
    rho = rng.random((BIG, BIG))
    rho *= 0.1
    rho += 0.3
    lat = B.Lattice(p)
    lat.init_rho(rho)
    lat.step(1)
    r1 = lat.rho()
    lat.close()
    del lat
    torch.cuda.empty_cache()
    corners = [(0, 0), (BIG - WIN, BIG - WIN), (BIG - WIN // 2, BIG - WIN // 2), (BIG // 2, BIG - WIN - 1),
               (17, BIG - WIN)]
    worst = 0.0
    for x0, y0 in corners:
        ys = (y0 + np.arange(WIN)) % BIG
        xs = (x0 + np.arange(WIN)) % BIG
        w0 = O.init_equilibrium(np.ascontiguousarray(rho[ys][:, xs]))
        O.step(w0, 1, p.G, p.tau)
        ro = O.density(w0)
        rg = r1[ys][:, xs]
        inner = (slice(MARGIN, WIN - MARGIN), slice(MARGIN, WIN - MARGIN))
        worst = max(worst, float(np.abs(rg[inner] - ro[inner]).max()))
    assert worst <= tol, worst

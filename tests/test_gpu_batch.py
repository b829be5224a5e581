"""Batched lattices: job table, segmented reductions, graph-replayed intervals,
admission against a device budget, retirement, fault isolation.

The central property: a job's result does not depend on what else is in the batch
(its reductions are decomposed by its own size only, and its FP16 dither follows its
own step count), so alone and in a mix its state is bit-identical.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

K = 20


def jobs_mix(storage, mlp=wl.MLP_F32):
    specs = [(64, 64, 1.0, -5.5), (96, 40, 0.9, -5.3), (130, 70, 1.0, -5.0), (200, 150, 1.1, -5.8),
             (61, 61, 1.0, -5.5), (256, 256, 0.95, -5.5)]
    out = []
    for k, (nx, ny, tau, G) in enumerate(specs):
        out.append(wl.Lattice(nx, ny, storage=storage, G=G, tau=tau, mlp=mlp,
                              droplets=[(nx / 2, ny / 2, min(nx, ny) / 4)], seed=40 + k, steps=100 * K, K=K))
    return out


def budget_for(jobs, max_jobs=64):
    return B.pl_batch_overhead_bytes(max_jobs) + sum(B.pl_batch_job_bytes(B.job_params(j)) for j in jobs) + (1 << 20)


@pytest.mark.parametrize("storage", [B.PL_F32, B.PL_F16_OFFSET])
def test_job_alone_and_in_mix_is_bit_identical(storage):
    jobs = jobs_mix(storage)
    blob = wl.mlp_weights(61)
    mix = B.Batch(storage, B.PL_MLP_F32, K, budget_for(jobs))
    mix.set_weights(blob)
    ids = [mix.submit(j) for j in jobs]
    assert all(i is not None for i in ids)
    mix.advance(3)
    for job, jid in zip(jobs, ids):
        alone = B.Batch(storage, B.PL_MLP_F32, K, budget_for([job]))
        alone.set_weights(blob)
        aid = alone.submit(job)
        alone.advance(3)
        fa, sa = alone.state(aid)
        fm, sm = mix.state(jid)
        assert sa == sm == 3 * K
        assert np.array_equal(fa, fm), (job.nx, job.ny)
        alone.close()
    mix.close()


def test_job_admitted_later_matches_alone():
    jobs = jobs_mix(B.PL_F16_OFFSET)
    blob = wl.mlp_weights(62)
    mix = B.Batch(B.PL_F16_OFFSET, B.PL_MLP_F32, K, budget_for(jobs))
    mix.set_weights(blob)
    first = mix.submit(jobs[0])
    mix.advance(2)
    late = mix.submit(jobs[3])            # joins after 2 intervals
    mix.advance(2)
    alone = B.Batch(B.PL_F16_OFFSET, B.PL_MLP_F32, K, budget_for([jobs[3]]))
    alone.set_weights(blob)
    aid = alone.submit(jobs[3])
    alone.advance(2)
    assert np.array_equal(alone.state(aid)[0], mix.state(late)[0])
    assert mix.state(first)[1] == 4 * K


def test_batch_matches_single_lattice_api():
    job = jobs_mix(B.PL_F32)[3]
    blob = wl.mlp_weights(63)
    bt = B.Batch(B.PL_F32, B.PL_MLP_F32, K, budget_for([job]))
    bt.set_weights(blob)
    jid = bt.submit(job)
    bt.advance(4)
    lat = B.Lattice(B.job_params(job))
    lat.init_droplets(job.droplets, job.rho_in, job.rho_out, job.width, job.noise_amp, job.seed)
    lat.set_weights(blob)
    lat.run(4 * K, K)
    assert np.array_equal(bt.state(jid)[0], lat.state()[0])


def test_batch_job_matches_oracle():
    job = jobs_mix(B.PL_F32)[1]
    blob = wl.mlp_weights(64)
    bt = B.Batch(B.PL_F32, B.PL_MLP_F32, K, budget_for([job]))
    bt.set_weights(blob)
    jid = bt.submit(job)
    bt.advance(5)
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    M0 = O.mass(f)
    assert O.run(f, 5 * K, job.G, job.tau, K=K, blob=blob, mode=O.MLP_F64, M0=M0) == 0
    ro = O.density(f)
    err = np.abs(O.density(bt.state(jid)[0]) - ro).max() / np.abs(ro).max()
    assert err < 1e-4, err


def test_retirement_results_and_budget():
    jobs = jobs_mix(B.PL_F16_OFFSET)[:3]
    blob = wl.mlp_weights(65)
    one = B.pl_batch_job_bytes(B.job_params(jobs[2]))
    # room for the largest job plus a little: the second submission must wait
    bt = B.Batch(B.PL_F16_OFFSET, B.PL_MLP_F32, K, B.pl_batch_overhead_bytes(8) + one + 4096, max_jobs=8)
    bt.set_weights(blob)
    a = bt.submit(jobs[2], steps=2 * K)
    assert a is not None
    assert bt.submit(jobs[2], steps=K) is None          # PL_ERR_BUDGET: no room now
    bt.advance(1)
    assert bt.poll() == []
    bt.advance(1)
    res = bt.poll()
    assert [r["id"] for r in res] == [a] and res[0]["steps"] == 2 * K and res[0]["status"] == 0
    m = res[0]["metrics"]
    # the correction projects the mass back to M0 and the FP16 mass restoration removes the
    # rounding of the apply pass to within one FP16 unit
    assert m["corrections"] == 2 and abs(m["mass"] - m["mass0"]) <= 1e-6 * m["mass0"]
    assert bt.info()["active"] == 0 and bt.info()["arena_used"] == 0
    b2 = bt.submit(jobs[2], steps=33)                    # now it fits; 33 steps round up to 2 K
    assert b2 is not None
    bt.advance(2)
    assert bt.poll()[0]["steps"] == 2 * K


def test_empty_batch_and_weights_order():
    """A batch refuses to advance before it has weights (PL_ERR_STATE); with weights and no job,
    advancing does nothing; a job submitted afterwards runs and retires as usual."""
    job = jobs_mix(B.PL_F32)[0]
    bt = B.Batch(B.PL_F32, B.PL_MLP_F32, K, budget_for([job], max_jobs=8), max_jobs=8)
    with pytest.raises(B.PLError) as e:
        bt.advance(1)
    assert e.value.status == B.PL_ERR_STATE
    bt.set_weights(job.weights())
    bt.advance(3)
    assert bt.poll() == [] and bt.info()["active"] == 0 and bt.info()["arena_used"] == 0
    jid = bt.submit(job, steps=K)
    assert jid is not None
    bt.advance(1)
    res = bt.poll()
    assert [r["id"] for r in res] == [jid] and res[0]["status"] == 0 and res[0]["steps"] == K
    assert res[0]["metrics"]["corrections"] == 1
    bt.close()


def test_fault_in_one_job_leaves_the_others_untouched():
    jobs = jobs_mix(B.PL_F32)[:3]
    bad = wl.Lattice(80, 80, storage=B.PL_F32, mlp=wl.MLP_F32, droplets=[(40.0, 40.0, 15.0)], rho_in=2.0,
                     rho_out=-0.5, seed=9, steps=100 * K, K=K)   # negative vapour density
    blob = wl.mlp_weights(66)
    mix = B.Batch(B.PL_F32, B.PL_MLP_F32, K, budget_for(jobs + [bad]))
    mix.set_weights(blob)
    ids = [mix.submit(j) for j in jobs]
    bid = mix.submit(bad, steps=2 * K)
    mix.advance(2)
    res = {r["id"]: r for r in mix.poll()}
    assert res[bid]["status"] == B.PL_ERR_NONPHYSICAL
    for job, jid in zip(jobs, ids):
        alone = B.Batch(B.PL_F32, B.PL_MLP_F32, K, budget_for([job]))
        alone.set_weights(blob)
        aid = alone.submit(job)
        alone.advance(2)
        assert np.array_equal(alone.state(aid)[0], mix.state(jid)[0])


def test_autotune_picks_a_candidate_and_keeps_results():
    jobs = jobs_mix(B.PL_F16_OFFSET)
    blob = wl.mlp_weights(67)
    a = B.Batch(B.PL_F16_OFFSET, B.PL_MLP_F32, K, budget_for(jobs))
    a.set_weights(blob)
    ids = [a.submit(j) for j in jobs]
    r = a.autotune(force=True)
    assert r in (8, 16, 24, 32, 48, 64, 96, 128)
    a.advance(2)
    b = B.Batch(B.PL_F16_OFFSET, B.PL_MLP_F32, K, budget_for(jobs))
    b.set_weights(blob)
    idb = [b.submit(j) for j in jobs]
    b.advance(2)
    for x, y, j in zip(ids, idb, jobs):
        assert np.array_equal(a.state(x)[0], b.state(y)[0])


def test_admission_into_retired_space_with_retune_matches_alone():
    """A job admitted into the arena space of a job that retired in the interval before, when
    the batch's total cell count moves to an octave the autotuner has not timed.  The retune's
    trial launches must run on the current job table: the table on the device still lists the
    retired 512^2 job, whose second population buffer now holds the new job's record and
    scratch (the new job, 384 x 256 FP16 cells, takes about 7.1 MB from offset 0, the old job's
    second buffer spans 5.2-10.5 MB).  The new job ends OK and bit-identical to its run alone."""
    storage = B.PL_F16_OFFSET
    big = wl.Lattice(512, 512, storage=storage, G=-5.5, tau=1.0, mlp=wl.MLP_F32,
                     droplets=[(256.0, 256.0, 80.0)], seed=71, steps=K, K=K)
    small = wl.Lattice(64, 64, storage=storage, G=-5.5, tau=1.0, mlp=wl.MLP_F32,
                       droplets=[(32.0, 32.0, 12.0)], seed=72, steps=6 * K, K=K)
    late = wl.Lattice(384, 256, storage=storage, G=-5.5, tau=1.0, mlp=wl.MLP_F32,
                      droplets=[(192.0, 128.0, 50.0)], seed=73, steps=3 * K, K=K)
    # the retired job's second population buffer: ten FP16 planes of 512 x 512 after the first
    buffer = 10 * 512 * 512 * 2
    assert buffer < B.pl_batch_job_bytes(B.job_params(late)) < 2 * buffer   # its record lies in it
    blob = wl.mlp_weights(63)
    bt = B.Batch(storage, B.PL_MLP_F32, K, budget_for([big, small]))
    bt.set_weights(blob)
    ib = bt.submit(big)
    bt.submit(small)
    bt.advance(1)
    assert [r["id"] for r in bt.poll()] == [ib]
    il = bt.submit(late)                  # first fit: the retired job's space
    assert il is not None
    bt.advance(3)
    done = {r["id"]: r for r in bt.poll()}
    assert done[il]["status"] == 0 and done[il]["steps"] == 3 * K, done[il]
    alone = B.Batch(storage, B.PL_MLP_F32, K, budget_for([late]))
    alone.set_weights(blob)
    aid = alone.submit(late)
    alone.advance(2)
    fa, sa = alone.state(aid)
    alone.close()
    bt2 = B.Batch(storage, B.PL_MLP_F32, K, budget_for([big, small]))
    bt2.set_weights(blob)
    bt2.submit(big)
    bt2.submit(small)
    bt2.advance(1)
    bt2.poll()
    il2 = bt2.submit(late)
    bt2.advance(2)
    fm, sm = bt2.state(il2)
    bt2.close()
    bt.close()
    assert sa == sm == 2 * K
    assert np.array_equal(fa, fm)


@pytest.mark.parametrize("storage", [B.PL_F32, B.PL_F16_OFFSET])
def test_interval_metrics_equal_a_fresh_metric_pass(storage):
    """A batch interval's metric pass reads the moment fields that the correction's apply pass
    leaves current (it skips its own moments pass).  Its records equal, bit for bit, those of a
    fresh metric pass of the same state (the single-lattice API, which recomputes the moments
    from the stored populations)."""
    job = jobs_mix(storage)[3]
    blob = wl.mlp_weights(65)
    bt = B.Batch(storage, B.PL_MLP_F32, K, budget_for([job]))
    bt.set_weights(blob)
    jid = bt.submit(job)
    bt.advance(4)
    live = {r["id"]: r for r in B.pl_batch_metrics(bt.h)}[jid]["metrics"]
    lat = B.Lattice(B.job_params(job))
    lat.init_droplets(job.droplets, job.rho_in, job.rho_out, job.width, job.noise_amp, job.seed)
    lat.set_weights(blob)
    lat.run(4 * K, K)
    assert np.array_equal(bt.state(jid)[0], lat.state()[0])
    fresh = lat.metrics()
    bt.close()
    for key in ("mass", "W", "G_max", "delta_rho", "W_eff", "E_int", "rho_max", "rho_min", "sum_g", "sum_g2",
                "count", "R_eq", "rho_in", "rho_out", "p_in", "p_out", "dP"):
        assert live[key] == fresh[key] or (np.isnan(live[key]) and np.isnan(fresh[key])), (key, live[key], fresh[key])

"""The density-stencil network variant (11 inputs) on the GPU against the oracle.

A variant that is not in the paper: the correction network reads the cell centre (x^, y^) and
the density of the cell and its 8 neighbours (velocity order c_0..c_8, periodic), so its field
depends on the state and is evaluated from the current density at every correction.  The
tolerances are those of the 2-input network: FP64 SIMT to rounding, FP32 SIMT 2e-5, the BF16
tensor-core kernel within 4e-3 of the oracle's BF16 emulation (see test_gpu_mlp_tc.py).
"""
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

DIMS = (11,) + wl.MLP_DIMS[1:]


def droplet_lattice(nx, ny, storage, mlp, **kw):
    p = B.pl_params_default(nx, ny, storage=storage, mlp=mlp, mlp_in=11, **kw)
    lat = B.Lattice(p)
    lat.init_droplets([(nx / 2, ny / 2, min(nx, ny) / 4), (0.2 * nx, 0.7 * ny, 3.0)], 2.0, 0.15, 2.0, 0.01, 4)
    lat.step(20)
    return lat


def test_blob_size_and_input_count_are_checked():
    assert B.pl_mlp_blob_size_for(11) == wl.mlp_blob_size(DIMS) == O.mlp_blob_size(11)
    assert B.pl_mlp_blob_size_for(2) == B.pl_mlp_blob_size()
    with pytest.raises(B.PLError):
        B.pl_mlp_blob_size_for(3)
    lat = droplet_lattice(32, 32, B.PL_F32, B.PL_MLP_F32)
    with pytest.raises(B.PLError):
        lat.set_weights(wl.mlp_weights(70))          # a 2-input blob for an 11-input lattice
    with pytest.raises(B.PLError):
        B.Lattice(B.pl_params_default(8, 8, mlp_in=5))


@pytest.mark.parametrize("storage,mlp,mode,tol", [
    (B.PL_F64, B.PL_MLP_F64, O.MLP_F64, 1e-13),
    (B.PL_F32, B.PL_MLP_F32, O.MLP_F64, 2e-5),
    (B.PL_F32, B.PL_MLP_BF16, O.MLP_BF16, 4e-3),
])
@pytest.mark.parametrize("nx,ny", [(64, 64), (67, 35), (300, 33)])
def test_stencil_network_field_matches_oracle(storage, mlp, mode, tol, nx, ny):
    blob = wl.mlp_weights(71, dims=DIMS)
    lat = B.Lattice(B.pl_params_default(nx, ny, storage=storage, mlp=mlp, mlp_in=11))
    drops = [(nx / 2, ny / 2, min(nx, ny) / 4), (0.2 * nx, 0.7 * ny, 3.0)]
    f = S.stored(S.oracle_droplet_state(nx, ny, drops, steps=20, seed=4), storage)
    lat.set_state(f, 20)
    lat.set_weights(blob)
    out = lat.mlp_field()
    ref = O.mlp_field(blob, nx, ny, mode, n_in=11, rho=O.density(f))
    assert np.isfinite(out).all()
    assert np.abs(out - ref).max() <= tol


def test_stencil_network_coupled_fp64_run_matches_oracle():
    job = wl.single_64()
    job.mlp_in, job.steps = 11, 400
    lat = B.Lattice.from_workload(job)
    lat.run(job.steps, job.K)
    f, _ = lat.state()
    m = lat.metrics()
    fo = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                       job.noise_amp, job.seed))
    M0 = O.mass(fo)
    assert O.run(fo, job.steps, job.G, job.tau, K=job.K, blob=job.weights(), mode=O.MLP_F64, M0=M0, n_in=11) == 0
    ro = O.density(fo)
    assert np.abs(lat.rho() - ro).max() / np.abs(ro).max() < 1e-11
    assert m["corrections"] == job.steps // job.K and abs(m["mass"] - M0) < 1e-12 * M0


def test_stencil_network_batch_alone_equals_mix_and_inputs_are_one_per_batch():
    K = 20
    jobs = [wl.Lattice(n, n, storage=wl.F16_OFFSET, mlp=wl.MLP_BF16, mlp_in=11, droplets=[(n / 2, n / 2, n / 4)],
                       seed=80 + n, steps=10 * K, K=K) for n in (48, 96, 130)]
    blob = jobs[0].weights()

    def batch(js):
        b = B.Batch(wl.F16_OFFSET, wl.MLP_BF16, K,
                    B.pl_batch_overhead_bytes(8) + sum(B.pl_batch_job_bytes(B.job_params(j)) for j in js) + (1 << 20),
                    max_jobs=8)
        b.set_weights(blob)
        return b, [b.submit(j) for j in js]

    mix, ids = batch(jobs)
    mix.advance(2)
    for j, jid in zip(jobs, ids):
        alone, (aid,) = batch([j])
        alone.advance(2)
        assert np.array_equal(alone.state(aid)[0], mix.state(jid)[0])
        alone.close()
    two = wl.Lattice(64, 64, storage=wl.F16_OFFSET, mlp=wl.MLP_BF16, droplets=[(32.0, 32.0, 10.0)], steps=K, K=K)
    with pytest.raises(B.PLError):
        mix.submit(two)                               # a 2-input job in an 11-input batch
    with pytest.raises(B.PLError):
        mix.set_weights(two.weights())
    mix.close()

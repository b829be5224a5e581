"""The correction's interface band (pl_params.mask_eps; the correction weighted toward the
interface, Sec. II-C, and adaptive sampling of the interface, Sec. IV-D; the band is this
library's reading): cells whose mask g / G_max is not above mask_eps are outside the interface
(mask 0), and the tensor-core network is evaluated on the compacted band only.

* FP64 lattices (FP64 CUDA-core network, every cell evaluated) against the oracle's band
  correction on the same state, to rounding (1e-13 of the largest population).
* The compacted tensor-core path: with a band threshold below every nonzero mask (1e-9) the
  band is every cell the full correction corrects, and each MMA row depends on its own operand
  row only, so the corrected state is bit-identical to mask_eps = 0 (the dense path).
* A real band (mask_eps = 0.05) with the BF16 network on FP32 storage: every cell outside the
  band (from the oracle's FP64 gradient; cells within FP32 rounding of the threshold aside) is
  left bit for bit, the state agrees with the oracle's band correction (BF16 emulation) within
  the network's rounding times the gains (1.5e-3 absolute), and the mass returns to M0.
* In a batch, a job with a band runs bit-identically alone and in a mix.
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


def seeded(nx, ny, storage, mlp, eps, seed=9):
    drops = [(nx / 2, ny / 2, min(nx, ny) / 4), (0.2 * nx, 0.3 * ny, 4.0)]
    f = S.stored(S.oracle_droplet_state(nx, ny, drops, steps=40, seed=seed), storage)
    lat = B.Lattice(B.pl_params_default(nx, ny, storage=storage, mlp=mlp, mask_eps=eps, beta_rho=0.3, beta_u=0.05))
    lat.set_state(f, 40)
    return lat, f


@pytest.mark.parametrize("eps", [0.01, 0.2])
@pytest.mark.parametrize("nx,ny", [(48, 48), (67, 35)])
def test_fp64_band_correction_matches_oracle(eps, nx, ny):
    lat, f0 = seeded(nx, ny, B.PL_F64, B.PL_MLP_F64, eps)
    blob = wl.mlp_weights(42)
    lat.set_weights(blob)
    lat.correct()
    f1, _ = lat.state()
    fo = f0.copy()
    assert O.correct(fo, blob, 0.3, 0.05, O.mass(f0), O.MLP_F64, eps=eps) == 0
    assert np.abs(f1 - fo).max() <= 1e-13 * np.abs(fo).max()
    g = O.grad_mag(O.density(f0))
    outside = (g / g.max()) <= eps
    assert np.array_equal(f1[:, outside], f0[:, outside])
    assert lat.metrics()["corrections"] == 1


@pytest.mark.parametrize("storage", [B.PL_F32, B.PL_F16_OFFSET])
@pytest.mark.parametrize("nx,ny", [(96, 80), (130, 70)])
def test_compacted_band_equals_dense_when_it_holds_every_cell(storage, nx, ny):
    blob = wl.mlp_weights(43)
    out = []
    for eps in (0.0, 1e-9):
        lat, _ = seeded(nx, ny, storage, B.PL_MLP_BF16, eps)
        lat.set_weights(blob)
        lat.correct()
        out.append(lat.state()[0])
        lat.close()
    assert np.array_equal(out[0], out[1])


def test_tensor_core_band_correction_against_oracle():
    nx, ny, eps = 96, 80, 0.05
    lat, f0 = seeded(nx, ny, B.PL_F32, B.PL_MLP_BF16, eps)
    m0 = lat.metrics()
    blob = wl.mlp_weights(44)
    lat.set_weights(blob)
    lat.correct()
    f1, _ = lat.state()
    fo = f0.copy()
    assert O.correct(fo, blob, 0.3, 0.05, O.mass(f0), O.MLP_BF16, eps=eps) == 0
    assert np.abs(f1 - fo).max() <= 1.5e-3
    g = O.grad_mag(O.density(f0))
    m = g / g.max()
    outside = m <= eps * (1.0 - 1e-6)
    assert np.array_equal(f1[:, outside], f0[:, outside])
    assert 0.05 < np.mean(~outside) < 0.5
    m1 = lat.metrics()
    assert m1["corrections"] == 1 and abs(m1["mass"] - m0["mass0"]) <= 1e-6 * m0["mass0"]


def test_batch_job_with_band_alone_and_in_mix():
    K = 20
    mk = lambda n, eps, seed: wl.Lattice(n, n, storage=wl.F16_OFFSET, mlp=wl.MLP_BF16, mask_eps=eps,
                                         droplets=[(n / 2, n / 2, n / 4)], seed=seed, steps=4 * K, K=K)
    jobs = [mk(64, 0.0, 1), mk(96, 0.05, 2), mk(130, 0.02, 3)]
    blob = wl.mlp_weights(45)

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
    live = {r["id"]: r for r in B.pl_batch_metrics(mix.h)}
    for jid in ids:
        assert live[jid]["status"] == 0 and live[jid]["metrics"]["corrections"] == 2
    mix.close()

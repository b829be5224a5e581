"""Seeded network weights through the C ABI (pl_init_mlp_weights, pl_batch_init_mlp_weights)
against the oracle's seeded blob (oracle.mlp_init_weights, pinned on the CPU): the same FP32
bits, and a batch seeded on the device runs exactly as one given the oracle's blob."""
import numpy as np
import pytest

import oracle as O
from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("n_in,storage", [(2, B.PL_F32), (11, B.PL_F16_OFFSET), (2, B.PL_F64)])
@pytest.mark.parametrize("seed", [0, 13, 2 ** 64 - 1])
def test_seeded_weights_equal_the_oracle_bits(n_in, storage, seed):
    mlp = B.PL_MLP_F64 if storage == B.PL_F64 else B.PL_MLP_BF16
    lat = B.Lattice(B.pl_params_default(40, 24, storage=storage, mlp=mlp, mlp_in=n_in))
    lat.init_weights(seed)
    got = B.pl_get_mlp_weights(lat.h, B.pl_mlp_blob_size_for(n_in))
    ref = O.mlp_init_weights(seed, n_in=n_in)
    assert got.dtype == np.float32 and np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    lat.close()


def test_batch_seeded_weights_run_as_the_uploaded_blob():
    job = wl.Lattice(96, 80, storage=wl.F16_OFFSET, mlp=wl.MLP_BF16, droplets=[(48.0, 40.0, 20.0)], steps=40, K=20)
    budget = B.pl_batch_overhead_bytes(4) + B.pl_batch_job_bytes(B.job_params(job)) + (1 << 20)
    out = []
    for seeded in (True, False):
        bt = B.Batch(wl.F16_OFFSET, wl.MLP_BF16, 20, budget, max_jobs=4)
        if seeded:
            bt.init_weights(21)
        else:
            bt.set_weights(O.mlp_init_weights(21))
        jid = bt.submit(job, steps=60)
        bt.advance(2)
        out.append(bt.state(jid)[0])
        bt.close()
    assert np.array_equal(out[0], out[1])

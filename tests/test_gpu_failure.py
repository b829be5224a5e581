"""Failure detection without a GPU fault.

Device-side waits are bounded: a wait that nothing satisfies gives up after its limit
and the kernel reports PL_ERR_TIMEOUT to the host, and the context stays usable.  No
test here traps, faults or hangs the GPU: the expired wait is on an mbarrier that
nothing arrives on, with a 50 ms limit.
"""
import time

import numpy as np
import pytest

from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_reports_timeout():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    st = B.pl_selftest_wait_timeout(status.data_ptr(), 50_000_000)
    dt = time.perf_counter() - t0
    assert st == B.PL_ERR_TIMEOUT
    assert int(status.item()) == B.PL_ERR_TIMEOUT
    assert 0.04 <= dt < 5.0
    # the context is still usable: a small coupled run completes normally
    job = wl.Lattice(48, 40, storage=B.PL_F32, mlp=wl.MLP_BF16, droplets=[(24.0, 20.0, 8.0)], K=10)
    lat = B.Lattice.from_workload(job)
    lat.run(20, 10)
    m = lat.metrics()
    assert m["status"] == B.PL_OK and m["corrections"] == 2


def test_selftest_rejects_bad_arguments():
    assert B.pl_selftest_wait_timeout(0, 1000) == B.PL_ERR_INVALID_ARG
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert B.pl_selftest_wait_timeout(status.data_ptr(), 10 ** 10) == B.PL_ERR_INVALID_ARG


def test_nonphysical_state_is_flagged_by_the_metrics():
    # a lattice initialised with a negative density is reported, not silently evolved
    lat = B.Lattice(B.pl_params_default(32, 32, storage=B.PL_F32, mlp=B.PL_MLP_F32))
    lat.init_droplets([(16.0, 16.0, 6.0)], 2.0, -0.5, 2.0, 0.0, 1)
    assert lat.status() == B.PL_ERR_NONPHYSICAL
    good = B.Lattice(B.pl_params_default(32, 32, storage=B.PL_F32, mlp=B.PL_MLP_F32))
    good.init_droplets([(16.0, 16.0, 6.0)], 2.0, 0.15, 2.0, 0.0, 1)
    assert good.status() == B.PL_OK

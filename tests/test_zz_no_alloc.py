"""pl_metrics_noalloc: the metric reduction for callers that cannot allocate device memory.

A caller that cannot call cudaMalloc (for instance code running inside another
library's allocator callback, or a process that must not grow its device footprint)
cannot lend the library a scratch buffer.  pl_metrics_noalloc keeps its scratch in a
static device array instead; this file checks, through the C ABI, that it returns the
same record as pl_metrics on the same populations, on two calls in a row.  It is named
to be collected last, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import seeded_states as S
from paper_2504_10539_gb300 import binding as B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FIELDS = ("mass", "W", "G_max", "delta_rho", "W_eff", "E_int", "rho_max", "rho_min", "sum_g", "sum_g2")


def populations_on_device(f, storage, pitch):
    """The documented layout: 9 planes (FP16-offset: 10, the offsets and the reference
    densities) of ny rows of `pitch` elements, x fastest."""
    _, ny, nx = f.shape
    if storage == B.PL_F64:
        dt, vals = torch.float64, torch.from_numpy(f)
    elif storage == B.PL_F32:
        dt, vals = torch.float32, torch.from_numpy(f).float()
    else:
        h, r = S.encode_f16(f)
        dt, vals = torch.float16, torch.from_numpy(np.concatenate([h, r[None]]))
    buf = torch.zeros((vals.shape[0], ny, pitch), dtype=dt, device="cuda")
    buf[:, :, :nx] = vals.to("cuda")
    return buf


@pytest.mark.parametrize("storage", [B.PL_F64, B.PL_F32, B.PL_F16_OFFSET])
@pytest.mark.parametrize("nx,ny", [(64, 64), (67, 35), (300, 33)])
def test_noalloc_metrics_match_pl_metrics(storage, nx, ny):
    mlp = B.PL_MLP_F64 if storage == B.PL_F64 else B.PL_MLP_F32
    lat = B.Lattice(B.pl_params_default(nx, ny, storage=storage, mlp=mlp))
    # a state the lattice holds exactly, so the caller's buffer below holds the same values
    f = S.stored(S.oracle_droplet_state(nx, ny, [(nx / 2, ny / 2, min(nx, ny) / 4)], steps=30, seed=11), storage)
    lat.set_state(f, 30)
    ref = lat.metrics()
    pitch = (nx + 7) // 8 * 8 + 8          # any pitch >= nx is accepted
    buf = populations_on_device(f, storage, pitch)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    tol = 1e-12 if storage == B.PL_F64 else 1e-6
    for _ in range(2):                     # two calls in a row share the static scratch
        got = B.pl_metrics_noalloc(buf.data_ptr(), nx, ny, pitch, storage, 0.0, 0.01, stream.cuda_stream)
        assert got["count"] == ref["count"]
        for k in FIELDS:
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1.0), k


def test_noalloc_rejects_lattices_beyond_its_scratch():
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(B.PLError) as e:
        B.pl_metrics_noalloc(buf.data_ptr(), 2048, 1024, 2048, B.PL_F32, 0.0, 0.01, 0)
    assert e.value.status == B.PL_ERR_BUDGET

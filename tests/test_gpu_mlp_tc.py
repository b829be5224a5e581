"""tcgen05 BF16 network kernel vs the oracle's BF16 emulation and FP64 network.

The kernel rounds the operands of layers 2-4 (weights and tanh outputs) to
BF16, accumulates in FP32 and uses the hardware tanh (relative error about
2^-11).  The oracle's BF16 mode rounds the same tensors to BF16 but uses exact
tanh and FP64 sums, so an activation can land one BF16 step (2^-8 relative)
apart where the exact value sits near a rounding boundary.  With weights drawn
in +-1/sqrt(fan_in) each layer damps such a step by about 1/sqrt(3); the bound
used below, 4e-3 absolute on outputs of size ~0.5, is a few such steps, and the
FP64 network differs from either by the BF16 rounding itself (<= 2e-2).
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

TOL_EMU = 4e-3
TOL_F64 = 2e-2


def field_lattice(nx, ny, storage=B.PL_F32):
    p = B.pl_params_default(nx, ny, storage=storage, mlp=B.PL_MLP_BF16)
    lat = B.Lattice(p)
    lat.init_droplets([], 1.0, 1.0, 2.0, 0.0, 1)
    return lat


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 7), (64, 64), (67, 35), (300, 33), (128, 3)])
@pytest.mark.parametrize("seed", [51, 52])
def test_bf16_network_field_matches_oracle(nx, ny, seed):
    blob = wl.mlp_weights(seed)
    lat = field_lattice(nx, ny)
    lat.set_weights(blob)
    out = lat.mlp_field()
    emu = O.mlp_field(blob, nx, ny, O.MLP_BF16)
    ref = O.mlp_field(blob, nx, ny, O.MLP_F64)
    assert np.isfinite(out).all()
    assert np.abs(out - emu).max() <= TOL_EMU
    assert np.abs(out - ref).max() <= TOL_F64
    assert lat.status() == B.PL_OK


def test_bf16_network_repeatable_and_weight_updates_take_effect():
    lat = field_lattice(96, 40)
    lat.set_weights(wl.mlp_weights(53))
    a = lat.mlp_field()
    b = lat.mlp_field()
    assert np.array_equal(a, b)
    lat.set_weights(wl.mlp_weights(54))
    c = lat.mlp_field()
    assert np.abs(c - O.mlp_field(wl.mlp_weights(54), 96, 40, O.MLP_BF16)).max() <= TOL_EMU


def test_bf16_network_special_weights():
    # zero weights: output = b5 exactly; single path: composition of four tanh
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    blob[-3:] = [0.5, -0.25, 0.125]
    lat = field_lattice(33, 17)
    lat.set_weights(blob)
    out = lat.mlp_field()
    assert np.array_equal(out[0], np.full((17, 33), 0.5))
    assert np.array_equal(out[2], np.full((17, 33), 0.125))


@pytest.mark.parametrize("side", [4096])
def test_bf16_network_full_size_sampled(side):
    """Full 4096x4096 field, every tile of the persistent grid; sampled cells vs the
    oracle evaluated one by one."""
    blob = wl.mlp_weights(55)
    lat = field_lattice(side, side, storage=B.PL_F16_OFFSET)
    lat.set_weights(blob)
    out = lat.mlp_field()
    assert np.isfinite(out).all()
    rng = np.random.default_rng(7)
    idx = rng.integers(0, side * side, size=3000)
    idx = np.concatenate([idx, [0, side - 1, side * side - 1, side * (side - 1)]])
    for c in idx:
        y, x = divmod(int(c), side)
        xh, yh = 2 * (x + 0.5) / side - 1, 2 * (y + 0.5) / side - 1
        e = O.mlp_forward(blob, xh, yh, O.MLP_BF16)
        assert np.abs(out[:, y, x] - e).max() <= TOL_EMU, (x, y)


def test_fp32_coupled_run_with_bf16_network_matches_emulating_oracle():
    n = 128
    job = wl.Lattice(n, n, storage=B.PL_F32, droplets=[(64.0, 64.0, 20.0)], seed=5, steps=600, K=100,
                     mlp=wl.MLP_BF16, weight_seed=15)
    lat = B.Lattice.from_workload(job)
    lat.run(job.steps, job.K)
    f_gpu, _ = lat.state()
    m = lat.metrics()
    fo = O.init_equilibrium(O.init_rho(n, n, job.droplets, 2.0, 0.15, 2.0, 0.01, 5))
    M0 = O.mass(fo)
    assert O.run(fo, job.steps, job.G, job.tau, K=job.K, blob=job.weights(), mode=O.MLP_BF16, M0=M0) == 0
    ro = O.density(fo)
    err = np.abs(O.density(f_gpu) - ro).max() / np.abs(ro).max()
    assert err < 1e-4, err
    assert m["corrections"] == 6 and m["status"] == 0
    assert abs(m["mass"] - M0) < 1e-6 * M0

"""The metric reductions (Sec. II-D Eqs. 9-13 as discretised in Sec. IV-E Eqs. 14-16, the mass,
and the Laplace measurement) of every storage type against the FP64 oracle on the same state.

The state is the oracle's droplet after 30 of its own steps, moved onto a grid on which each
cell's density is the same number in the kernels' FP32 (or FP64) and in the oracle's FP64
(seeded_states.exact_state), and loaded with pl_set_state.  With equal densities, what is
left is the kernels' own arithmetic, so the bounds are tight:
  - mass: the FP32 per-block error-free pair sums carry ~48 bits, the FP64 folds 53:
    1e-12 relative;
  - rho_max, rho_min: equal (FP64 lattices: the kernel sums a cell's populations pairwise,
    the oracle in order: a few FP64 roundings);
  - |grad rho| per cell (FP32 lattices): gx, gy exact, then one rounding of gx^2 + gy^2 and
    one of the square root: within 2^-23 relative, so sum g, G_max within 2^-22 and
    sum g^2 (E_int) within 2^-21 of the oracle's, W_eff within 2^-20;
  - the count of W: equal up to the cells whose oracle gradient is within 2^-22 of the
    threshold (none here, as it happens, but the bound is the definition);
  - Laplace fields (one centred droplet): R_eq, rho_in, rho_out 1e-9 relative (FP32 region
    distances: no cell here lies within FP32 rounding of a region boundary, checked);
    p_in, p_out within 1e-6 absolute (FP32 pseudopotential per cell).
A 1e-5 relative slip in a pair sum, a dropped cell, an off-by-one neighbour or a wrong
threshold comparison fails these.  pl_metrics_noalloc is held to the same bounds.
"""
import numpy as np
import pytest

import oracle as O
import seeded_states as S
from paper_2504_10539_gb300 import binding as B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SIZES = [(64, 64), (67, 35), (300, 33), (515, 260), (1024, 1024)]
THR = 0.01


def case(storage, nx, ny):
    drop = (nx / 2.0, ny / 2.0, 0.3 * min(nx, ny))
    f = S.exact_state(S.oracle_droplet_state(nx, ny, [drop], steps=30, seed=nx + 7 * ny), storage)
    mlp = B.PL_MLP_F64 if storage == S.F64 else B.PL_MLP_F32
    lat = B.Lattice(B.pl_params_default(nx, ny, storage=storage, mlp=mlp))
    lat.init_droplets([drop], 2.0, 0.15, 2.0, 0.01, 1)   # records the droplet centre (Laplace)
    lat.set_state(f, 30)
    assert np.array_equal(lat.state()[0], f)           # stored without rounding
    return lat, f, drop


def check_metric_record(m, rho, storage):
    mo = O.metrics_rho(rho, THR)
    exact = storage != S.F64
    rel_g = 2.0 ** -22 if exact else 1e-12
    assert abs(m["mass"] - mo["mass"]) <= 1e-12 * abs(mo["mass"])
    tol_r = 0.0 if exact else 1e-14
    for k in ("rho_max", "rho_min"):
        assert abs(m[k] - mo[k]) <= tol_r * abs(mo[k]), k
    assert abs(m["delta_rho"] - mo["delta_rho"]) <= 2 * tol_r * abs(mo["rho_max"]) + 1e-300
    for k, r in (("G_max", rel_g), ("sum_g", rel_g), ("sum_g2", 2 * rel_g), ("E_int", 2 * rel_g),
                 ("W_eff", 4 * rel_g)):
        assert abs(m[k] - mo[k]) <= r * abs(mo[k]) + 1e-12 * abs(mo[k]), (k, m[k], mo[k])
    g = O.grad_mag(rho)
    ambiguous = int(np.sum(np.abs(g - THR) <= rel_g * THR))
    assert abs(m["count"] - mo["count"]) <= ambiguous, (m["count"], mo["count"], ambiguous)
    assert m["W"] == m["count"] / rho.size


@pytest.mark.parametrize("storage", [S.F64, S.F32, S.F16])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_metrics_and_laplace_match_oracle_on_same_state(storage, nx, ny):
    lat, f, drop = case(storage, nx, ny)
    m = lat.metrics()
    rho = O.density(f)
    check_metric_record(m, rho, storage)
    lo = O.laplace(rho, drop[0], drop[1], 2.0, -5.5)
    if storage == S.F64:
        for k in ("R_eq", "rho_in", "rho_out", "p_in", "p_out", "dP"):
            assert abs(m[k] - lo[k]) <= 1e-11 * abs(lo[k]), k
    else:
        # no cell within FP32 rounding of a region boundary, so both sides use the same cells
        y, x = np.mgrid[0:ny, 0:nx]
        d = np.hypot(np.minimum(np.abs(x - drop[0]), nx - np.abs(x - drop[0])),
                     np.minimum(np.abs(y - drop[1]), ny - np.abs(y - drop[1])))
        for edge in (0.5 * lo["R_eq"], lo["R_eq"] + 8.0):   # 4 FP32 units of the distance
            assert np.min(np.abs(d - edge)) > 4.0 * 2.0 ** -23 * edge
        for k in ("R_eq", "rho_in", "rho_out"):
            assert abs(m[k] - lo[k]) <= 1e-9 * abs(lo[k]), k
        for k in ("p_in", "p_out", "dP"):
            assert abs(m[k] - lo[k]) <= 1e-6, k
    lat.close()


@pytest.mark.parametrize("storage", [S.F64, S.F32, S.F16])
@pytest.mark.parametrize("nx,ny", [(67, 35), (1024, 1024)])
def test_noalloc_metrics_match_oracle_on_same_state(storage, nx, ny):
    lat, f, _ = case(storage, nx, ny)
    lat.close()
    pitch = (nx + 7) // 8 * 8
    if storage == S.F64:
        dt, vals = torch.float64, torch.from_numpy(f)
    elif storage == S.F32:
        dt, vals = torch.float32, torch.from_numpy(f).float()
    else:                                   # ten planes: the offsets and the references
        h, r = S.encode_f16(f)
        dt, vals = torch.float16, torch.from_numpy(np.concatenate([h, r[None]]))
    buf = torch.zeros((vals.shape[0], ny, pitch), dtype=dt, device="cuda")
    buf[:, :, :nx] = vals.to("cuda")
    torch.cuda.synchronize()
    m = B.pl_metrics_noalloc(buf.data_ptr(), nx, ny, pitch, storage, 0.0, THR, 0)
    check_metric_record(m, O.density(f), storage)

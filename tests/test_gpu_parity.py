"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several CTA strips (126 owned columns each) and row blocks (32 rows)
with ragged tails, plus degenerate lattices (1x1, 2x3, 1xN).  Tolerances:
FP64 storage ~ 1e-12 relative (operation order only); FP32 storage 1e-4
relative L-infinity on rho (the target for FP32 storage); FP16-offset storage
bounded by the FP16 rounding of the stored offsets.
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

F64, F32, F16 = B.PL_F64, B.PL_F32, B.PL_F16_OFFSET
SIZES = [(1, 1), (2, 3), (1, 9), (5, 7), (67, 35), (130, 70), (300, 33)]


def lattice(nx, ny, storage, mlp=None, **kw):
    if mlp is None:
        mlp = B.PL_MLP_F64 if storage == F64 else B.PL_MLP_F32
    p = B.pl_params_default(nx, ny, storage=storage, mlp=mlp, **kw)
    return B.Lattice(p)


def stored(f, storage):
    """The FP64 values a storage type actually holds for populations f."""
    return S.stored(f, storage)


def rel_linf(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# ----------------------------------------------------------------------------- initial state

@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_init_droplets_matches_oracle(storage, nx, ny):
    drops = [(nx / 2, ny / 2, min(nx, ny) / 4), (0.3 * nx, 0.8 * ny, 2.5)]
    lat = lattice(nx, ny, storage)
    lat.init_droplets(drops, 2.0, 0.15, 2.0, 0.01, 7)
    f, step = lat.state()
    fo = O.init_equilibrium(O.init_rho(nx, ny, drops, 2.0, 0.15, 2.0, 0.01, 7))
    assert step == 0
    tol = {F64: 2e-15, F32: 1e-7, F16: 3e-4}[storage]
    assert np.abs(f - fo).max() <= tol
    if storage == F32:
        assert np.array_equal(f, stored(fo, F32))


# ----------------------------------------------------------------------------- one step

@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_step_matches_oracle(storage, nx, ny, tau):
    f0 = stored(wl.random_populations(nx, ny, seed=nx * 1000 + ny, lo=0.02, hi=0.3), storage)
    lat = lattice(nx, ny, storage, tau=tau, G=-5.5)
    lat.set_state(f0, 0)
    assert np.array_equal(lat.state()[0], f0)
    lat.step(3)
    f, step = lat.state()
    fo = f0.copy()
    O.step(fo, 3, -5.5, tau)
    assert step == 3
    tol = {F64: 1e-13, F32: 2e-6, F16: 2e-3}[storage]
    assert np.abs(f - fo).max() <= tol * np.abs(fo).max()


# ----------------------------------------------------------------------------- degenerate cases

@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_uniform_fluid_at_rest_stays_at_rest(storage):
    """A uniform density at rest is a fixed point of Eq. 1 (zero force, equilibrium populations),
    and a stable one below the critical coupling (G = -3 against -4 for this pseudopotential;
    inside the spinodal, e.g. rho = 0.7 at G = -5.5, rounding noise grows into phase
    separation, as it must): after 50 steps every cell's density is the initial one and its
    momentum zero, to the storage's rounding (FP16: offsets of a rest state against per-cell
    references are a fixed small value, rounded stochastically each step)."""
    nx, ny, rho0 = 40, 24, 0.7
    lat = lattice(nx, ny, storage, G=-3.0, tau=0.9)
    lat.init_rho(np.full((ny, nx), rho0))
    lat.step(50)
    f, _ = lat.state()
    rho = f.sum(axis=0)
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7])
    jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8])
    tol = {F64: 1e-14, F32: 1e-6, F16: 2e-5}[storage]
    assert np.abs(rho - rho0).max() <= tol * rho0
    assert max(np.abs(jx).max(), np.abs(jy).max()) <= tol * rho0
    m = lat.metrics()
    assert m["status"] == 0 and m["W"] == 0.0


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_correction_without_an_interface_changes_nothing(storage):
    """A uniform field has no density gradient: G_max = 0, the mask m is 0 in every cell, and
    the correction (Sec. II-C, as the oracle reads it) changes no population and reports OK,
    in the oracle and on the GPU alike."""
    nx, ny = 40, 24
    blob = wl.mlp_weights(42)
    lat = lattice(nx, ny, storage)
    lat.init_rho(np.full((ny, nx), 0.7))
    lat.set_weights(blob)
    f0, step0 = lat.state()
    lat.correct()
    f1, step1 = lat.state()
    assert step1 == step0 and np.array_equal(f1, f0)
    assert lat.status() == 0
    fo = f0.copy()
    assert O.correct(fo, blob, 0.1, 0.01, O.mass(f0), O.MLP_F64) == 0
    assert np.array_equal(fo, f0)


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_no_interaction_droplet_matches_oracle(storage):
    """G = 0: no Shan-Chen force, the droplet only relaxes and diffuses (no phase separation);
    20 steps against the oracle.  Tolerances of the three-step test above, the FP16 one scaled
    by sqrt(20 / 3) for the stochastic rounding of every step accumulating as a random walk."""
    nx, ny = 48, 40
    f0 = stored(S.oracle_droplet_state(nx, ny, [(24.0, 20.0, 9.0)], steps=0, seed=5), storage)
    lat = lattice(nx, ny, storage, G=0.0, tau=1.0)
    lat.set_state(f0, 0)
    lat.step(20)
    f, _ = lat.state()
    fo = f0.copy()
    O.step(fo, 20, 0.0, 1.0)
    tol = {F64: 1e-13, F32: 2e-6, F16: 2e-3 * (20 / 3) ** 0.5}[storage]
    assert np.abs(f - fo).max() <= tol * np.abs(fo).max()


# ----------------------------------------------------------------------------- coupled droplet runs

def test_single_64_fp64_coupled_run_matches_oracle():
    """64x64 FP64 droplet, 2000 steps, FP64 network correction every 50 steps."""
    job = wl.single_64()
    lat = B.Lattice.from_workload(job)
    lat.run(job.steps, job.K)
    m = lat.metrics()
    f_gpu, step = lat.state()
    fo = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                       job.noise_amp, job.seed))
    M0 = O.mass(fo)
    assert O.run(fo, job.steps, job.G, job.tau, K=job.K, blob=job.weights(), mode=O.MLP_F64,
                 beta_rho=job.beta_rho, beta_u=job.beta_u, M0=M0) == 0
    ro = O.density(fo)
    assert step == 2000 and m["corrections"] == 40 and m["status"] == 0
    assert rel_linf(lat.rho(), ro) < 1e-11
    mo = O.metrics_rho(ro)
    lo = O.laplace(ro, 32.0, 32.0, job.width, job.G)
    assert abs(m["mass"] - M0) < 1e-12 * M0 and abs(mo["mass"] - M0) < 1e-12 * M0
    assert m["count"] == mo["count"]
    for k in ("G_max", "W_eff", "E_int", "delta_rho"):
        assert abs(m[k] - mo[k]) <= 1e-10 * abs(mo[k]), k
    for k in ("R_eq", "rho_in", "rho_out", "p_in", "p_out", "dP"):
        assert abs(m[k] - lo[k]) <= 1e-9 * abs(lo[k]), k


def test_fp32_droplet_with_fp32_network_matches_oracle():
    n = 128
    job = wl.Lattice(n, n, storage=F32, droplets=[(64.0, 64.0, 20.0)], seed=5, steps=600, K=100,
                     mlp=wl.MLP_F32, weight_seed=15)
    lat = B.Lattice.from_workload(job)
    lat.run(job.steps, job.K)
    m = lat.metrics()
    f_gpu, _ = lat.state()
    fo = O.init_equilibrium(O.init_rho(n, n, job.droplets, 2.0, 0.15, 2.0, 0.01, 5))
    M0 = O.mass(fo)
    assert O.run(fo, job.steps, job.G, job.tau, K=job.K, blob=job.weights(), mode=O.MLP_F64, M0=M0) == 0
    assert rel_linf(lat.rho(), O.density(fo)) < 1e-4
    assert abs(m["mass"] - M0) < 1e-6 * M0
    mo = O.metrics_rho(O.density(fo))
    assert abs(m["W"] - mo["W"]) <= 0.02 * mo["W"]


# ----------------------------------------------------------------------------- metrics, network, correction

@pytest.mark.parametrize("storage,mode,tol", [(F64, B.PL_MLP_F64, 1e-13), (F32, B.PL_MLP_F32, 2e-5)])
@pytest.mark.parametrize("nx,ny", [(64, 64), (67, 35)])
def test_network_field_matches_oracle(storage, mode, tol, nx, ny):
    blob = wl.mlp_weights(41)
    lat = lattice(nx, ny, storage, mlp=mode)
    lat.init_droplets([], 1.0, 1.0, 2.0, 0.0, 1)
    lat.set_weights(blob)
    out = lat.mlp_field()
    ref = O.mlp_field(blob, nx, ny, O.MLP_F64)
    assert np.abs(out - ref).max() <= tol


@pytest.mark.parametrize("storage,tol", [(F64, 1e-13), (F32, 2e-5)])
def test_single_correction_matches_oracle(storage, tol):
    n = 48
    lat = lattice(n, n, storage, beta_rho=0.3, beta_u=0.05)
    f0 = stored(S.oracle_droplet_state(n, n, [(24.0, 24.0, 10.0)], steps=40, seed=9), storage)
    lat.set_state(f0, 40)
    m0 = lat.metrics()
    blob = wl.mlp_weights(42)
    lat.set_weights(blob)
    lat.correct()
    f1, _ = lat.state()
    fo = f0.copy()
    assert O.correct(fo, blob, 0.3, 0.05, O.mass(f0), O.MLP_F64) == 0
    assert np.abs(f1 - fo).max() <= tol * np.abs(fo).max()
    m1 = lat.metrics()
    assert m1["corrections"] == 1 and m1["status"] == 0
    assert abs(m1["mass"] - m0["mass0"]) <= (1e-12 if storage == F64 else 1e-6) * m0["mass0"]


@pytest.mark.parametrize("nx,ny", [(48, 48), (67, 35), (130, 70)])
def test_f16_correction_matches_oracle_and_restores_mass(nx, ny):
    """FP16-offset storage: the correction of the stored state agrees with the oracle's
    correction of the same (decoded) state to the FP16 rounding of the stored offsets, and
    the stored mass returns to M0 within 1e-6 (the rest offsets absorb the rounding of the
    moving ones; every offset is rounded stochastically, and offsets are small, so that
    rounding is too)."""
    lat = lattice(nx, ny, F16, beta_rho=0.3, beta_u=0.05)
    f0 = stored(S.oracle_droplet_state(nx, ny, [(nx / 2, ny / 2, min(nx, ny) / 4)], steps=40, seed=9), F16)
    lat.set_state(f0, 40)
    m0 = lat.metrics()
    blob = wl.mlp_weights(42)
    lat.set_weights(blob)
    lat.correct()
    f1, _ = lat.state()
    fo = f0.copy()
    assert O.correct(fo, blob, 0.3, 0.05, O.mass(f0), O.MLP_F64) == 0
    # Per cell, in offset space h = f - Wr_i r(x - c_i) (stored as 2^10 h; the references of the stored state,
    # which the correction leaves as they are): every offset is rounded stochastically (less
    # than one FP16 spacing); the rest population takes the cell's corrected mass minus the
    # rounded moving populations, so their eight rounding errors land in it before its own.
    _, r = S.encode_f16(f0)
    off = S.WREF[:, None, None] * S.source_refs(r.astype(np.float64))
    # FP16 spacing of the stored (2^10-scaled) offsets, in population units
    sp = np.maximum(np.spacing((np.abs(fo - off) * S.SCALE).astype(np.float16)),
                    np.spacing((np.abs(f1 - off) * S.SCALE).astype(np.float16)))
    sp = sp.astype(np.float64) / S.SCALE             # the larger spacing if the two straddle a binade
    # The corrected values themselves differ from the oracle's by the FP32 network (within
    # 2e-5 of the FP64 one) times beta_rho = 0.3, i.e. < 1e-5: near a rounding midpoint that
    # can tip a rounding, hence the slack.
    slack = 1e-5
    err = np.abs(f1 - fo)
    assert np.all(err[1:] <= sp[1:] + slack)
    assert np.all(err[0] <= sp[0] + err[1:].sum(axis=0) + slack)
    m1 = lat.metrics()
    assert m1["corrections"] == 1 and m1["status"] == 0
    assert abs(m1["mass"] - m0["mass0"]) <= 1e-6 * m0["mass0"]


def test_nonphysical_correction_leaves_state_and_sets_status():
    n = 32
    lat = lattice(n, n, F64, beta_rho=1.0, beta_u=0.0)
    f0 = S.oracle_droplet_state(n, n, [(16.0, 16.0, 6.0)], steps=20, seed=1)
    lat.set_state(f0, 20)
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    offs, o = [], 0
    dims = wl.MLP_DIMS
    for l in range(5):
        offs.append(o)
        o += dims[l + 1] * dims[l] + dims[l + 1]
    for l, w in enumerate([2.0, 1.0, 1.0, 1.0, 200.0]):
        blob[offs[l]] = w
    lat.set_weights(blob)
    lat.correct()
    assert lat.status() == B.PL_ERR_NONPHYSICAL
    assert np.array_equal(lat.state()[0], f0)
    fo = f0.copy()
    assert O.correct(fo, blob, 1.0, 0.0, O.mass(f0)) == -4


# ----------------------------------------------------------------------------- determinism, checkpoint

@pytest.mark.parametrize("storage", [F32, F16])
def test_repeat_runs_are_bit_identical(storage):
    job = wl.Lattice(96, 80, storage=storage, droplets=[(40.0, 40.0, 15.0)], seed=2, K=25, mlp=wl.MLP_F32)
    outs = []
    for _ in range(2):
        lat = B.Lattice.from_workload(job)
        lat.run(120, 25)
        outs.append((lat.state()[0], lat.metrics()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("storage", [F64, F32])
def test_checkpoint_resume_is_exact(storage):
    job = wl.Lattice(70, 40, storage=storage, droplets=[(30.0, 20.0, 9.0)], seed=4, K=10,
                     mlp=wl.MLP_F64 if storage == F64 else wl.MLP_F32)
    a = B.Lattice.from_workload(job)
    a.run(30, 10)
    a.run(30, 10)
    b = B.Lattice.from_workload(job)
    b.run(30, 10)
    f_mid, step = b.state()
    c = B.Lattice.from_workload(job)   # fresh lattice, weights loaded, state overwritten
    c.set_state(f_mid, step)
    c.run(30, 10)
    assert np.array_equal(a.state()[0], c.state()[0])
    assert c.state()[1] == 60


def test_run_schedule_equals_explicit_steps_and_corrections():
    job = wl.Lattice(40, 40, storage=F64, droplets=[(20.0, 20.0, 8.0)], seed=6, K=7, mlp=wl.MLP_F64)
    a = B.Lattice.from_workload(job)
    a.run(23, 7)
    b = B.Lattice.from_workload(job)
    for s in range(1, 24):
        b.step(1)
        if s % 7 == 0:
            b.correct()
    assert np.array_equal(a.state()[0], b.state()[0])
    assert a.metrics()["corrections"] == 3

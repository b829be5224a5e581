"""Network training on the GPU (Eqs. 3-8, Adam) against the training oracle.

FP64 lattices train in FP64: the gradient, the loss terms and the trained weights agree
with the oracle to rounding (the weights are the FP64 results rounded to FP32 on both
sides, so they may differ by one FP32 unit).  FP32 and FP16-offset lattices train in FP32:
each sample's gradient passes through five layers and three tangent rows in FP32 (a few
units of 2^-24 relative each) and is summed over all cells in a fixed order, so the
gradient is compared with a bound of 1e-4 of its largest component.  Adam divides by
sqrt(v) + eps, which turns a rounding difference in a near-zero gradient component into a
step of up to lr; the multi-epoch FP32 comparison therefore runs with eps = 1e-2, where
the update is Lipschitz in the gradient with constant lr / eps, and the default eps is
checked through the loss history.
"""
import numpy as np
import pytest

import oracle as O
import oracle.train as T
import seeded_states as S
from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HP = {
    "default": {},
    "phys": dict(lambda_phys=3e3, lambda_int=0.0),
    "int": dict(lambda_phys=0.0, lambda_int=1e3, alpha2=50.0),
}


def droplet_lattice(nx, ny, storage, steps=40, seed=3):
    """A lattice holding the oracle's droplet after `steps` of its steps (stored exactly in the
    lattice's storage type); returns the lattice, its job and that state, which both sides read."""
    mlp = B.PL_MLP_F64 if storage == B.PL_F64 else B.PL_MLP_BF16
    job = wl.Lattice(nx, ny, storage=storage, mlp=mlp, droplets=[(nx / 2, ny / 2, min(nx, ny) / 4)], seed=seed,
                     K=1, weight_seed=30 + seed)
    f = S.stored(S.oracle_droplet_state(nx, ny, job.droplets, steps=steps, G=job.G, tau=job.tau, seed=seed), storage)
    lat = B.Lattice(B.job_params(job))
    lat.set_state(f, steps)
    lat.set_weights(job.weights())
    return lat, job, f


def oracle_gradient(f, job, hp):
    t, iface = T.targets_from_state(f, 0.01)
    L, terms, g = T.loss_and_grad(job.weights(), job.nx, job.ny, t, iface, job.G, 1.0, T.TrainParams(**hp))
    return L, terms, g


@pytest.mark.parametrize("which", sorted(HP))
@pytest.mark.parametrize("nx,ny", [(64, 64), (37, 23), (300, 33), (5, 3)])
def test_fp64_gradient_matches_oracle(nx, ny, which):
    lat, job, f = droplet_lattice(nx, ny, B.PL_F64)
    tr = B.Trainer(lat, max_epochs=4, **HP[which])
    g, loss = tr.gradient()
    L, terms, go = oracle_gradient(f, job, HP[which])
    assert np.isfinite(g).all()
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()
    assert loss[0] == pytest.approx(L, rel=1e-11)
    for k in range(3):
        assert loss[1 + k] == pytest.approx(terms[k], rel=1e-10, abs=1e-300)


@pytest.mark.parametrize("storage", [B.PL_F32, B.PL_F16_OFFSET])
@pytest.mark.parametrize("which", sorted(HP))
@pytest.mark.parametrize("nx,ny", [(64, 64), (67, 35)])
def test_fp32_gradient_matches_oracle(nx, ny, which, storage):
    lat, job, f = droplet_lattice(nx, ny, storage)
    tr = B.Trainer(lat, max_epochs=4, **HP[which])
    g, loss = tr.gradient()
    t, iface = T.targets_from_state(f, 0.01)
    # The GPU decides the interface set (Eq. 16 gradient > 0.01) from an FP32 density: a cell
    # whose FP64 gradient lies within FP32 rounding of the threshold may fall on either side,
    # and both results are correct.  Accept the oracle gradient of any such assignment.
    gm = O.grad_mag(O.density(f)).ravel()
    amb = np.flatnonzero(np.abs(gm - 0.01) < 2e-6)
    assert amb.size <= 3
    ok = []
    for bits in range(1 << amb.size):
        m = iface.copy()
        m[amb] = [(bits >> q) & 1 == 1 for q in range(amb.size)]
        L, _, go = T.loss_and_grad(job.weights(), job.nx, job.ny, t, m, job.G, 1.0, T.TrainParams(**HP[which]))
        ok.append(np.abs(g - go).max() <= 1e-4 * np.abs(go).max() and abs(loss[0] - L) <= 1e-5 * abs(L))
    assert any(ok)


def test_fp64_training_matches_oracle_and_persists_adam_state():
    lat, job, f = droplet_lattice(48, 40, B.PL_F64)
    tr = B.Trainer(lat, max_epochs=8)
    blob1, hist1, st = T.train(job.weights(), f, 5, job.G)
    tr.train(5)
    w1 = lat.weights().astype(np.float64)
    assert np.all(np.abs(w1 - blob1) <= np.abs(blob1.astype(np.float64)) * 2.0 ** -23)
    assert np.abs(tr.losses(5) - hist1).max() <= 1e-10 * np.abs(hist1).max()
    # a second call continues Adam (steps 6..8) from the FP32 blob
    blob2, hist2, st = T.train(lat.weights(), f, 3, job.G, state=st)
    tr.train(3)
    assert np.abs(lat.weights().astype(np.float64) - blob2).max() <= 2.0 ** -23 * np.abs(blob2).max()
    assert np.abs(tr.losses(3) - hist2).max() <= 1e-10 * np.abs(hist2).max()


@pytest.mark.parametrize("storage", [B.PL_F32, B.PL_F16_OFFSET])
def test_fp32_training_matches_oracle(storage):
    lat, job, f = droplet_lattice(64, 48, storage)
    # well-conditioned Adam (eps = 1e-2): weights within 10 epochs x lr/eps x gradient error
    tr = B.Trainer(lat, max_epochs=10, eps=1e-2)
    tr.train(10)
    blob, hist, _ = T.train(job.weights(), f, 10, job.G, hp=T.TrainParams(eps=1e-2))
    assert np.abs(lat.weights().astype(np.float64) - blob).max() <= 1e-6
    assert np.abs(tr.losses(10) - hist).max() <= 1e-5 * np.abs(hist).max()
    # default eps: the loss history follows the oracle's
    lat2, _, _ = droplet_lattice(64, 48, storage)
    tr2 = B.Trainer(lat2, max_epochs=10)
    tr2.train(10)
    _, hist2, _ = T.train(job.weights(), f, 10, job.G)
    assert np.abs(tr2.losses(10)[:, 0] - hist2[:, 0]).max() <= 1e-4 * hist2[0, 0]


def test_fp64_coupled_run_with_training_matches_oracle():
    job = wl.Lattice(48, 48, storage=B.PL_F64, mlp=B.PL_MLP_F64, droplets=[(24.0, 24.0, 10.0)], seed=5, K=20,
                     weight_seed=41)
    lat = B.Lattice.from_workload(job)
    tr = B.Trainer(lat, max_epochs=4)
    tr.run(50, 20, 3)                                   # 2 rounds (steps 20, 40) and 10 plain steps
    f, step = lat.state()
    m = lat.metrics()
    fo = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                       job.noise_amp, job.seed))
    M0 = O.mass(fo)
    st, blob, _ = T.run_trained(fo, 50, job.G, job.tau, 20, job.weights(), 3, M0=M0)
    assert st == 0 and step == 50
    ro = O.density(fo)
    assert np.abs(lat.rho() - ro).max() <= 1e-10 * np.abs(ro).max()
    assert np.abs(lat.weights().astype(np.float64) - blob).max() <= 2.0 ** -23 * np.abs(blob).max()
    assert m["corrections"] == 2 and abs(m["mass"] - M0) <= 1e-12 * M0


def test_trainer_argument_and_state_checks():
    p = B.pl_params_default(32, 32, storage=B.PL_F32)
    lat = B.Lattice(p)
    tr = B.Trainer(lat, max_epochs=3)
    with pytest.raises(B.PLError) as e:
        tr.train(1)                                     # no state, no weights
    assert e.value.status == B.PL_ERR_STATE
    lat.init_droplets([(16.0, 16.0, 6.0)], 2.0, 0.15, 2.0, 0.01, 1)
    with pytest.raises(B.PLError):
        tr.train(1)                                     # no weights
    lat.set_weights(wl.mlp_weights(3))
    for bad in (0, 4):
        with pytest.raises(B.PLError) as e:
            tr.train(bad)
        assert e.value.status == B.PL_ERR_INVALID_ARG
    tr.train(3)
    with pytest.raises(B.PLError):
        tr.losses(4)
    assert tr.losses(3).shape == (3, 4)
    with pytest.raises(B.PLError):
        B.Trainer(lat, max_epochs=3, lr=-1.0)
    lat11 = B.Lattice(B.pl_params_default(16, 16, mlp_in=11))
    with pytest.raises(B.PLError):
        B.Trainer(lat11)


def test_full_size_512_gradient_matches_oracle():
    """The 512 x 512 single-droplet lattice (FP32 storage), after 200 steps: the full-batch
    gradient and loss terms against the oracle's over all 262,144 cells."""
    job = wl.single_512()
    f = S.stored(S.oracle_droplet_state(job.nx, job.ny, job.droplets, steps=200, G=job.G, tau=job.tau, seed=job.seed),
                 job.storage)
    lat = B.Lattice(B.job_params(job))
    lat.set_state(f, 200)
    lat.set_weights(job.weights())
    tr = B.Trainer(lat, max_epochs=2)
    g, loss = tr.gradient()
    L, terms, go = oracle_gradient(f, job, {})
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
    assert loss[0] == pytest.approx(L, rel=1e-5)
    tr.train(2)
    h = tr.losses(2)
    assert h[1, 0] < h[0, 0]


def test_protocol_series_match_oracle():
    """Sec. III-C protocol on a 48 x 48 FP64 droplet (shortened: 60 initial steps recorded
    every 20, rounds of 20 steps with 4, 3, 2 epochs): every recorded metric of the initial,
    PINN-LBM and pure-LBM series against the oracle running the same sequence."""
    from paper_2504_10539_gb300 import protocol
    job = wl.Lattice(48, 48, storage=B.PL_F64, mlp=B.PL_MLP_F64, droplets=[(24.0, 24.0, 10.0)], seed=6, K=20,
                     weight_seed=42)
    out = protocol.run(job, init_steps=60, K=20, epochs=(4, 3, 2), record_every=20)
    assert out["status"] == {"pinn": 0, "pure": 0}
    fo = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                       job.noise_amp, job.seed))
    M0 = O.mass(fo)

    def close(gpu, f):
        ref = O.metrics_rho(O.density(f))
        for k in protocol.METRICS:
            assert gpu[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-12), k

    close(out["init"][0][1], fo)
    for step, m in out["init"][1:]:
        O.step(fo, 20, job.G, job.tau)
        close(m, fo)
    fp = fo.copy()
    blob, st = job.weights(), None
    for (step, e, m, losses), (step2, mp) in zip(out["pinn"], out["pure"]):
        O.step(fo, 20, job.G, job.tau)
        blob, hist, st = T.train(blob, fo, e, job.G, state=st)
        assert O.correct(fo, blob, job.beta_rho, job.beta_u, M0, O.MLP_F64) == 0
        O.step(fp, 20, job.G, job.tau)
        close(m, fo)
        close(mp, fp)
        assert losses[0] == pytest.approx(hist[0, 0], rel=1e-10) and losses[1] == pytest.approx(hist[-1, 0], rel=1e-10)
    assert [e for _, e, _, _ in out["pinn"]] == [4, 3, 2] and out["pinn"][-1][0] == 120


@pytest.mark.parametrize("storage,mlp,mode,tol", [(B.PL_F32, B.PL_MLP_F32, O.MLP_F64, 1e-4),
                                                   (B.PL_F16_OFFSET, B.PL_MLP_BF16, O.MLP_BF16, 1e-2)])
def test_coupled_run_with_training_fp32_arithmetic(storage, mlp, mode, tol):
    """FP32 / FP16-offset lattices with FP32 training, two coupled rounds against the FP64
    oracle (FP32 storage with the FP32 network; FP16 storage with the BF16 tensor-core network
    and the oracle's BF16 emulation); the relative L-inf bounds on rho are the ones the storage
    types are held to (1e-4 FP32, 1e-2 FP16)."""
    job = wl.Lattice(64, 64, storage=storage, mlp=mlp, droplets=[(32.0, 32.0, 12.0)], seed=7, K=25,
                     weight_seed=43)
    lat = B.Lattice.from_workload(job)
    tr = B.Trainer(lat, max_epochs=4, eps=1e-2)
    tr.run(50, 25, 4)
    f, _ = lat.state()
    m = lat.metrics()
    fo = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                       job.noise_amp, job.seed))
    M0 = O.mass(fo)
    st, blob, _ = T.run_trained(fo, 50, job.G, job.tau, 25, job.weights(), 4, hp=T.TrainParams(eps=1e-2), mode=mode,
                                M0=M0)
    assert st == 0 and m["status"] == 0 and m["corrections"] == 2
    ro = O.density(fo)
    assert np.abs(lat.rho() - ro).max() <= tol * np.abs(ro).max()
    # the correction restores the lattice's own M0 (the mass of its stored initial state)
    assert abs(m["mass"] - m["mass0"]) <= 1e-6 * m["mass0"]

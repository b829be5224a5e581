"""Tensor-core training (PL_TRAIN_TC) against the FP64 training oracle.

Layers 2-4 of the forward pass, of the reverse pass and of the weight gradient, and the bias
and layer-1 gradients, run as BF16 tcgen05 MMAs with FP32 accumulation: the activations, their
tangents, the back-propagated gradients, the weights and the sample coordinates enter each MMA
rounded to BF16 (2^-9 relative).  A gradient entry
sums one product of two such operands per sample and row, so its error is a few 2^-9 of the
magnitudes it sums; the bound used is 2e-2 of the largest gradient component, and the loss
(whose forward pass has three BF16 layers) is held to 1e-2 relative.
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


def seeded_lattice(job, steps):
    """A lattice holding the oracle's droplet of `job` after `steps` of its steps (stored exactly
    in the lattice's storage type), with the job's weights; returns the lattice and the state."""
    f = S.stored(S.oracle_droplet_state(job.nx, job.ny, job.droplets, steps=steps, G=job.G, tau=job.tau,
                                        seed=job.seed), job.storage)
    lat = B.Lattice(B.job_params(job))
    lat.set_state(f, steps)
    lat.set_weights(job.weights())
    return lat, f


def droplet_lattice(nx, ny, storage=B.PL_F32, steps=40, seed=3):
    job = wl.Lattice(nx, ny, storage=storage, mlp=B.PL_MLP_BF16, droplets=[(nx / 2, ny / 2, min(nx, ny) / 4)],
                     seed=seed, K=1, weight_seed=30 + seed)
    lat, f = seeded_lattice(job, steps)
    return lat, job, f


def oracle_gradient(f, job, hp, iface=None):
    t, m = T.targets_from_state(f, 0.01)
    return T.loss_and_grad(job.weights(), job.nx, job.ny, t, m if iface is None else iface, job.G, 1.0,
                           T.TrainParams(**hp))


# relative to the largest component of the FP64 oracle's gradient (of the block, per layer)
GRAD_TOL = 5 * 2.0 ** -9


@pytest.mark.parametrize("which", sorted(HP))
@pytest.mark.parametrize("nx,ny", [(64, 64), (67, 35), (41, 7)])
def test_tc_gradient_matches_oracle(nx, ny, which):
    lat, job, f = droplet_lattice(nx, ny)
    tr = B.Trainer(lat, max_epochs=2, mode=B.PL_TRAIN_TC, **HP[which])
    g, loss = tr.gradient()
    L, terms, go = oracle_gradient(f, job, HP[which])
    assert np.isfinite(g).all()
    err = np.abs(g - go).max() / np.abs(go).max()
    # BF16 operands (2^-9 relative each); the longest chain of rounded operands on the way to a
    # weight gradient is five (forward 2-4, reverse 4-3), 5 x 2^-9 ~ 1e-2 (measured up to 4.7e-3)
    assert err <= GRAD_TOL, err
    assert loss[0] == pytest.approx(L, rel=1e-2)


def test_tc_gradient_per_layer_blocks():
    """Each layer's block of the gradient on its own (a wrong operand layout in one MMA shows
    up as a block far from the oracle even when the whole vector's maximum is dominated by
    another layer)."""
    lat, job, f = droplet_lattice(96, 80)
    tr = B.Trainer(lat, max_epochs=1, mode=B.PL_TRAIN_TC)
    g, _ = tr.gradient()
    _, _, go = oracle_gradient(f, job, {})
    sizes = [(64, 2), (64,), (128, 64), (128,), (128, 128), (128,), (64, 128), (64,), (3, 64), (3,)]
    o = 0
    for shp in sizes:
        n = int(np.prod(shp))
        blk, ref = g[o:o + n], go[o:o + n]
        assert np.abs(blk - ref).max() <= GRAD_TOL * np.abs(ref).max() + 1e-12, (shp, o)
        o += n
    assert o == g.size


def test_tc_training_follows_oracle_and_full_size():
    lat, job, f = droplet_lattice(64, 48)
    tr = B.Trainer(lat, max_epochs=10, mode=B.PL_TRAIN_TC)
    tr.train(10)
    h = tr.losses(10)
    _, hist, _ = T.train(job.weights(), f, 10, job.G)
    assert np.abs(h[:, 0] - hist[:, 0]).max() <= 2e-2 * hist[0, 0]
    assert h[-1, 0] < h[0, 0]
    # the 512 x 512 single droplet: one gradient over all 262,144 cells
    big = wl.single_512()
    lat2, f2 = seeded_lattice(big, 100)
    tr2 = B.Trainer(lat2, max_epochs=1, mode=B.PL_TRAIN_TC)
    g, loss = tr2.gradient()
    L, _, go = oracle_gradient(f2, big, {})
    assert np.abs(g - go).max() <= GRAD_TOL * np.abs(go).max()
    assert loss[0] == pytest.approx(L, rel=1e-2)


def test_tc_gradient_is_reproducible():
    """The gradient is a fixed-order sum: TMEM accumulation over a CTA's tiles in tile order, one
    writer per element of a CTA's slice, the slices folded in CTA order; two calls on the same
    state give the same bits (also for a lattice whose last tile is partial)."""
    for nx, ny in [(96, 80), (67, 35)]:
        lat, job, _ = droplet_lattice(nx, ny)
        tr = B.Trainer(lat, max_epochs=2, mode=B.PL_TRAIN_TC)
        g1, l1 = tr.gradient()
        g2, l2 = tr.gradient()
        assert np.array_equal(g1, g2) and np.array_equal(l1, l2), (nx, ny)
        tr.close()
        lat.close()


def test_tc_coupled_run_and_mode_checks():
    job = wl.Lattice(64, 64, storage=B.PL_F16_OFFSET, mlp=B.PL_MLP_BF16, droplets=[(32.0, 32.0, 12.0)], seed=7, K=25,
                     weight_seed=43)
    lat = B.Lattice.from_workload(job)
    tr = B.Trainer(lat, max_epochs=4, mode=B.PL_TRAIN_TC)
    tr.run(50, 25, 4)
    m = lat.metrics()
    assert m["status"] == 0 and m["corrections"] == 2
    assert abs(m["mass"] - m["mass0"]) <= 1e-6 * m["mass0"]
    lat64 = B.Lattice(B.pl_params_default(16, 16, storage=B.PL_F64, mlp=B.PL_MLP_F64))
    with pytest.raises(B.PLError):
        B.Trainer(lat64, mode=B.PL_TRAIN_TC)


def test_protocol_with_tensor_core_training_follows_fp32_training():
    """The Sec. III-C protocol (shortened) with either training form: the BF16 tensor-core
    training moves the weights by steps that differ from the FP32 ones only through the BF16
    rounding of the gradient, so every recorded interface metric agrees closely."""
    from paper_2504_10539_gb300 import protocol
    job = wl.Lattice(96, 96, storage=B.PL_F32, mlp=B.PL_MLP_F32, droplets=[(48.0, 48.0, 16.0)], seed=8, K=20,
                     weight_seed=44)
    a = protocol.run(job, init_steps=60, K=20, epochs=(20, 10), record_every=30)
    b = protocol.run(job, init_steps=60, K=20, epochs=(20, 10), record_every=30, hyper=dict(mode=B.PL_TRAIN_TC))
    assert a["status"] == b["status"] == {"pinn": 0, "pure": 0}
    for (s1, e1, m1, l1), (s2, e2, m2, l2) in zip(a["pinn"], b["pinn"]):
        assert (s1, e1) == (s2, e2)
        for k in protocol.METRICS:
            assert m2[k] == pytest.approx(m1[k], rel=1e-3, abs=1e-9), k
        assert l2[0] == pytest.approx(l1[0], rel=1e-2) and l2[1] == pytest.approx(l1[1], rel=2e-2)
    assert a["pure"] == b["pure"]

"""The seeded workload generators against the recipes they state (no GPU).

The benchmark, the parity tests and the oracle all draw their inputs from
``paper_2504_10539_gb300.workloads``; these checks pin the shapes, ranges and structure
of what it draws (sizes, parameter ranges, droplet placement, arrival process), its
determinism per seed, and its one table of derived physics (the Shan-Chen coexistence
densities of served jobs) against scipy root finding on the scheme's equation of state.
"""
import numpy as np
import pytest

from paper_2504_10539_gb300 import workloads as wl


def test_batch_256_recipe():
    jobs = wl.batch_256()
    assert len(jobs) == 256
    # the benchmark's unit count: one step of the batch updates this many cells
    assert sum(j.cells for j in jobs) == 101_896_192
    seeds = set()
    for j in jobs:
        assert j.nx == j.ny and j.nx % 64 == 0 and 64 <= j.nx <= 1024
        assert -6.0 <= j.G <= -5.0
        # tau uniform in [0.6, 1.2], restricted to the scheme's stable part for the lattice's G
        assert max(0.6, wl.tau_min_stable(j.G)) <= j.tau <= 1.2
        assert len(j.droplets) == 1
        cx, cy, r = j.droplets[0]
        assert (cx, cy) == (j.nx / 2.0, j.ny / 2.0)
        assert 0.1 * j.nx <= r <= 0.35 * j.nx
        assert (j.storage, j.mlp, j.K, j.steps) == (wl.F16_OFFSET, wl.MLP_BF16, 100, 2000)
        assert (j.rho_in, j.rho_out) == (2.0, 0.15)
        seeds.add(j.seed)
    assert len(seeds) == 256                                    # every lattice its own noise
    assert len({j.weight_seed for j in jobs}) == 1              # one network for the batch
    # the draws cover their ranges (not a degenerate generator)
    sides = np.array([j.nx for j in jobs])
    assert sides.min() == 64 and sides.max() == 1024 and len(set(sides)) == 16
    Gs = np.array([j.G for j in jobs])
    assert Gs.min() < -5.9 and Gs.max() > -5.1


def test_batch_256_is_deterministic_and_seed_dependent():
    a, b, c = wl.batch_256(n=32), wl.batch_256(n=32), wl.batch_256(n=32, seed=5)
    assert [(j.nx, j.G, j.tau, j.droplets, j.seed) for j in a] == [(j.nx, j.G, j.tau, j.droplets, j.seed) for j in b]
    assert [(j.nx, j.G) for j in a] != [(j.nx, j.G) for j in c]
    assert len(wl.batch_256(n=8)) == 8


def test_tau_stability_table():
    # the measured bounds at the table points, monotone in -G, clamped outside
    for g, t in zip(wl.TAU_STABLE_G, wl.TAU_STABLE_MIN):
        assert wl.tau_min_stable(-g) == pytest.approx(t)
    ts = [wl.tau_min_stable(-g) for g in np.linspace(5.0, 6.0, 41)]
    assert all(x <= y for x, y in zip(ts, ts[1:]))
    assert wl.tau_min_stable(-4.0) == wl.TAU_STABLE_MIN[0] and wl.tau_min_stable(-7.0) == wl.TAU_STABLE_MIN[-1]


def test_field_4096_recipe():
    for storage in (wl.F16_OFFSET, wl.F32):
        job = wl.field_4096(storage=storage)
        assert (job.nx, job.ny, job.storage, job.tau, job.G) == (4096, 4096, storage, 0.8, -5.5)
        assert (job.steps, job.K, job.mlp) == (5000, 100, wl.MLP_BF16)
        assert (job.rho_in, job.rho_out) == (wl.FIELD_RHO_IN, wl.FIELD_RHO_OUT)
        assert len(job.droplets) == 400
        d = np.array(job.droplets)
        assert (d[:, 0] >= 0).all() and (d[:, 0] < 4096).all() and (d[:, 1] >= 0).all() and (d[:, 1] < 4096).all()
        assert d[:, 2].min() >= 8.0 and d[:, 2].max() <= 40.0
    # both storages see the same field; the accuracy crop keeps the droplet density
    assert wl.field_4096(storage=wl.F32).droplets == wl.field_4096(storage=wl.F16_OFFSET).droplets
    crop = wl.field_4096(storage=wl.F32, side=512, n_drop=400 * 512 * 512 // (4096 * 4096))
    assert (crop.nx, len(crop.droplets)) == (512, 6)


def test_serve_poisson_recipe():
    reqs = wl.serve_poisson()
    assert len(reqs) == 500
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # exponential inter-arrival times at 200 per second: mean 5 ms (500 draws: within 15%),
    # coefficient of variation near 1
    assert gaps.mean() == pytest.approx(1 / 200, rel=0.15)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, abs=0.15)
    for r in reqs:
        j = r.job
        assert j.nx == j.ny and j.nx % 32 == 0 and 64 <= j.nx <= 2048
        assert 1 <= len(j.droplets) <= 8
        for cx, cy, rad in j.droplets:
            assert 0 <= cx < j.nx and 0 <= cy < j.ny and 6.0 <= rad <= max(6.0, 0.3 * j.nx)
        assert -6.0 <= j.G <= -5.0 and j.tau == wl.serve_tau(j.G)
        assert (j.rho_out, j.rho_in) == wl.coexistence(j.G)
        assert 1000 <= j.steps <= 20000 and j.K == 100 and j.storage == wl.F16_OFFSET
    assert len({r.job.seed for r in reqs}) == 500


def test_serve_tau():
    assert wl.serve_tau(-5.0) == 1.0 and wl.serve_tau(-5.5) == 1.0
    assert wl.serve_tau(-6.0) == pytest.approx(1.2)
    assert wl.serve_tau(-5.75) == pytest.approx(1.1)


def _coexistence(G):
    """Shan-Chen mechanical-stability coexistence of p = rho/3 + G psi^2/6, psi = 1 - exp(-rho):
    p(rho_v) = p(rho_l) and int_{rho_v}^{rho_l} (p0 - p) psi'/psi^2 drho = 0."""
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    psi = lambda r: 1.0 - np.exp(-r)
    p = lambda r: r / 3 + G * psi(r) ** 2 / 6

    def eqs(v):
        rv, rl = v
        p0 = p(rv)
        return [p(rl) - p0, quad(lambda r: (p0 - p(r)) * np.exp(-r) / psi(r) ** 2, rv, rl)[0]]

    return fsolve(eqs, [0.1, 2.3], xtol=1e-12)


@pytest.mark.parametrize("k", range(11))
def test_coexistence_table_solves_the_shan_chen_conditions(k):
    G = -wl.COEX_G[k]
    rv, rl = _coexistence(G)
    # the table holds four decimals
    assert abs(wl.COEX_VAPOUR[k] - rv) < 6e-5, (G, rv)
    assert abs(wl.COEX_LIQUID[k] - rl) < 6e-5, (G, rl)
    assert wl.coexistence(G) == (wl.COEX_VAPOUR[k], wl.COEX_LIQUID[k])


def test_mlp_weights_ranges_and_determinism():
    w = wl.mlp_weights(11)
    assert w.dtype == np.float32 and w.size == wl.mlp_blob_size() == 33475
    assert np.array_equal(w, wl.mlp_weights(11)) and not np.array_equal(w, wl.mlp_weights(12))
    off = 0
    dims = wl.MLP_DIMS
    for l in range(len(dims) - 1):
        nin, nout = dims[l], dims[l + 1]
        bound = 1.0 / np.sqrt(nin)
        part = w[off:off + nout * nin + nout]
        assert np.abs(part).max() <= bound * (1 + 1e-7)
        assert np.abs(part).max() > 0.9 * bound                  # the range is used
        off += nout * nin + nout
    assert off == w.size
    z = wl.mlp_weights(11, zero_bias=True)
    assert z[64 * 2:64 * 2 + 64].tolist() == [0.0] * 64         # b1

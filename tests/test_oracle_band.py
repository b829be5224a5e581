"""Pins of the oracle's interface band (the correction's emphasis on the interface, Sec. II-C;
adaptive sampling of the interface, Sec. IV-D; reading: cells whose mask g / G_max is not above
eps are outside the interface and get mask 0).  Checked against what the definition fixes:
  - the corrected cells are exactly the band {m > eps}: every other cell is left bit for bit;
  - the projections still return the total mass to M0 and keep the total momentum, whatever
    eps (a projection over the wrong set breaks one of them);
  - eps >= 1 leaves no cell in the band (the identity), and the band shrinks as eps grows.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_10539_gb300 import workloads as wl


def state(n=48, steps=30):
    f = O.init_equilibrium(O.init_rho(n, n, [(n / 2, n / 2, n / 4), (10.0, 12.0, 4.0)], 2.0, 0.15, 2.0, 0.01, 5))
    M0 = O.mass(f)
    O.step(f, steps, -5.5, 1.0)
    return f, M0


def band(f, eps):
    g = O.grad_mag(O.density(f))
    return (g / g.max()) > eps


@pytest.mark.parametrize("eps", [0.0, 0.01, 0.1, 0.4])
def test_band_cells_are_exactly_the_corrected_ones(eps):
    f, M0 = state()
    blob = wl.mlp_weights(5)
    f1 = f.copy()
    assert O.correct(f1, blob, 0.3, 0.05, M0, eps=eps) == 0
    inside = band(f, eps)
    changed = np.any(f1 != f, axis=0)
    assert not np.any(changed & ~inside)
    assert np.mean(changed[inside]) > 0.99


@pytest.mark.parametrize("eps", [0.0, 0.05, 0.3])
def test_band_projection_keeps_mass_at_M0_and_momentum(eps):
    f, M0 = state()
    blob = wl.mlp_weights(6)
    jx0, jy0 = O.momentum(f)
    f1 = f.copy()
    assert O.correct(f1, blob, 0.3, 0.05, M0, eps=eps) == 0
    assert abs(O.mass(f1) - M0) <= 1e-13 * M0
    jx1, jy1 = O.momentum(f1)
    scale = np.abs(jx0).sum() + np.abs(jy0).sum() + 1.0
    assert abs(jx1.sum() - jx0.sum()) <= 1e-13 * scale and abs(jy1.sum() - jy0.sum()) <= 1e-13 * scale


def test_band_above_one_is_the_identity_and_shrinks_with_eps():
    f, M0 = state()
    blob = wl.mlp_weights(7)
    f1 = f.copy()
    assert O.correct(f1, blob, 0.3, 0.05, M0, eps=1.0) == 0
    assert np.array_equal(f1, f)
    sizes = [band(f, e).sum() for e in (0.0, 0.01, 0.1, 0.5)]
    assert sizes == sorted(sizes, reverse=True) and sizes[0] > sizes[-1] > 0


def test_coupled_run_with_band_conserves_mass():
    f, M0 = state(steps=0)
    assert O.run(f, 60, -5.5, 1.0, K=20, blob=wl.mlp_weights(8), eps=0.05, M0=M0) == 0
    assert abs(O.mass(f) - M0) <= 1e-12 * M0

"""Pins of the oracle's seeded network weights (the configurations' "seed-initialised"
network of Sec. III-B; the reading: entry k of the blob is (2 U(seed, k) - 1)/sqrt(fan_in),
U the SplitMix64 uniform of output k, rounded to FP32).

* The first five entries for seed 1234567 follow from the published SplitMix64 outputs
  (tests/golden/splitmix64_seed1234567.txt) and the layer-1 fan-in of 2, worked out here
  from those integers alone.
* Every layer's entries, scaled by sqrt(fan_in), are uniform on [-1, 1): range, mean and
  variance per layer, which fail if a layer took another layer's fan-in or the blob's
  segments were misaligned.
"""
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DIMS = (2, 64, 128, 128, 64, 3)


def segments(n_in):
    dims = (n_in,) + DIMS[1:]
    k = 0
    for l in range(5):
        n = dims[l + 1] * dims[l] + dims[l + 1]
        yield dims[l], k, k + n
        k += n


def test_first_entries_follow_the_published_generator_outputs():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    w = O.mlp_init_weights(1234567)
    for k, v in enumerate(vals):
        u = (v >> 11) / 2.0 ** 53
        assert w[k] == np.float32((2.0 * u - 1.0) / np.sqrt(2.0)), k


def test_blob_length_and_layer_distributions():
    for n_in in (2, 11):
        w = O.mlp_init_weights(77, n_in=n_in).astype(np.float64)
        assert w.size == O.mlp_blob_size(n_in)
        for fan_in, a, b in segments(n_in):
            s = w[a:b] * np.sqrt(fan_in)
            n = b - a
            assert s.min() >= -1.0 - 1e-6 and s.max() <= 1.0 + 1e-6, (n_in, fan_in)
            if n >= 1000:   # a wrong fan-in moves the extremes by a factor >= sqrt(2)
                assert s.max() > 0.98 and s.min() < -0.98, (n_in, fan_in)
            assert abs(s.mean()) < 5.0 * np.sqrt(1.0 / 3.0 / n), (n_in, fan_in)
            assert abs(s.var() - 1.0 / 3.0) < 6.0 * np.sqrt(4.0 / 45.0 / n), (n_in, fan_in)


def test_seeds_differ_and_repeat():
    a, b = O.mlp_init_weights(5), O.mlp_init_weights(6)
    assert np.array_equal(a, O.mlp_init_weights(5))
    assert np.mean(a == b) < 1e-3

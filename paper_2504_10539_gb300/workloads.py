"""Seeded synthetic inputs for the droplet workloads.

This module only draws numbers: droplet centres and radii, per-lattice
parameters, network weights and request arrival times.  It holds none of the
method's arithmetic (no profile, no step, no metric); the CUDA path and the
CPU oracle each take these inputs and compute from them independently.

The workloads follow the droplet set-up of Sec. III-A of the paper (periodic
square box, one droplet, density ratio, tau = 1.0, g = -5.5) and the network of
Sec. III-B, scaled to the five lattice configurations this library is measured
on:

* ``single_64``   : 64x64, FP64, one droplet R=12, 2000 steps, correction every 50.
* ``single_512``  : 512x512, FP32, one droplet R=80, 10000 steps, correction every 100.
* ``field_4096``  : 4096x4096, FP16-offset (and FP32), 400 droplets R~U[8,40],
                    tau=0.8, 5000 steps, correction every 100.
* ``batch_256``   : 256 lattices, side U{64..1024}, G~U[-6,-5], tau~U[0.6,1.2],
                    one centred droplet R~U[0.1,0.35]*side, 2000 steps, FP16-offset.
* ``serve_poisson``: Poisson arrivals at 200/s, side U{64..2048 step 32}, 1-8
                    droplets R~U[6, 0.3*side], G~U[-6,-5] (tau from ``serve_tau``, started
                    at the coexistence densities of G), steps U[1000,20000], correction
                    every 100, 150 GB device budget.

Random draws use numpy's PCG64 generator seeded per workload.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

# Storage codes shared with the C ABI header (PL_F64, PL_F32, PL_F16_OFFSET).
F64, F32, F16_OFFSET = 0, 1, 2
# Network arithmetic codes (PL_MLP_F64, PL_MLP_F32, PL_MLP_BF16).
MLP_F64, MLP_F32, MLP_BF16 = 0, 1, 2

# Layer widths of the network of Sec. III-B: 2 -> 64 -> 128 -> 128 -> 64 -> 3.
MLP_DIMS = (2, 64, 128, 128, 64, 3)


def mlp_blob_size(dims=MLP_DIMS) -> int:
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def mlp_weights(seed: int, dims=MLP_DIMS, zero_bias: bool = False) -> np.ndarray:
    """FP32 weight blob W1,b1,...,W5,b5 (row-major W[out][in]) with every entry
    drawn uniformly in [-1/sqrt(fan_in), +1/sqrt(fan_in)], layer by layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        nin, nout = dims[l], dims[l + 1]
        bound = 1.0 / np.sqrt(nin)
        parts.append(rng.uniform(-bound, bound, size=nout * nin))
        b = rng.uniform(-bound, bound, size=nout)
        parts.append(np.zeros(nout) if zero_bias else b)
    return np.concatenate(parts).astype(np.float32)


@dataclasses.dataclass
class Lattice:
    """One periodic droplet lattice: geometry, physics, initial state recipe."""
    nx: int
    ny: int
    storage: int = F32
    G: float = -5.5
    tau: float = 1.0
    rho0: float = 1.0
    mask_eps: float = 0.0             # interface band of the correction (0: every cell)
    droplets: List[Tuple[float, float, float]] = dataclasses.field(default_factory=list)
    rho_in: float = 2.0
    rho_out: float = 0.15
    width: float = 2.0
    noise_amp: float = 0.01
    seed: int = 1                     # noise seed (counter-based, per cell)
    steps: int = 0
    K: int = 0                        # correction interval, 0 = none
    mlp: int = MLP_F32
    weight_seed: int = 11
    beta_rho: float = 0.1
    beta_u: float = 0.01
    mlp_in: int = 2                   # network inputs: 2 = (x^, y^); 11 = with the density stencil

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def weights(self) -> np.ndarray:
        return mlp_weights(self.weight_seed, dims=(self.mlp_in,) + MLP_DIMS[1:])


def single_64(seed: int = 1) -> Lattice:
    return Lattice(64, 64, storage=F64, droplets=[(32.0, 32.0, 12.0)], seed=seed, steps=2000, K=50,
                   mlp=MLP_F64, weight_seed=10 + seed)


def single_512(seed: int = 2) -> Lattice:
    return Lattice(512, 512, storage=F32, droplets=[(256.0, 256.0, 80.0)], seed=seed, steps=10000,
                   K=100, mlp=MLP_BF16, weight_seed=10 + seed)


def field_droplets(n: int, nx: int, ny: int, rmin: float, rmax: float, seed: int):
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, nx, size=n)
    cy = rng.uniform(0.0, ny, size=n)
    r = rng.uniform(rmin, rmax, size=n)
    return [(float(a), float(b), float(c)) for a, b, c in zip(cx, cy, r)]


# Coexistence densities of the scheme at G = -5.5, tau = 0.8 (plateaus of a relaxed
# flat interface).  The field starts there: started from 2.0 / 0.15, the relaxation
# transient at tau = 0.8 drives the vapour density negative within 100 steps.
FIELD_RHO_IN, FIELD_RHO_OUT = 2.2727, 0.0743


def field_4096(storage: int = F16_OFFSET, seed: int = 3, side: int = 4096, n_drop: int = 400) -> Lattice:
    return Lattice(side, side, storage=storage, tau=0.8,
                   droplets=field_droplets(n_drop, side, side, 8.0, 40.0, 100 + seed),
                   rho_in=FIELD_RHO_IN, rho_out=FIELD_RHO_OUT,
                   seed=seed, steps=5000, K=100, mlp=MLP_BF16, weight_seed=10 + seed)


# Stability of the scheme for a droplet started at 2.0 / 0.15 (the batch's initial state):
# smallest tau (step 0.05) at which FP64 oracle runs of 2000 steps on 256x256, with one
# centred droplet of radius 0.1 and 0.35 of the side, kept every density positive and
# finite.  Small droplets are the less stable ones: G = -5 -> 0.65, -5.25 -> 0.8, -5.5 ->
# 0.85, -5.75 -> 0.9, -6 -> 0.95 (large droplets: 0.6, 0.7, 0.8, 0.85, 0.9).  Below it the
# relaxation transient drives the vapour density negative within a few hundred steps.
TAU_STABLE_G = (5.0, 5.25, 5.5, 5.75, 6.0)          # -G
TAU_STABLE_MIN = (0.70, 0.85, 0.90, 0.95, 1.00)     # the small-droplet bound + 0.05


def tau_min_stable(G: float) -> float:
    """Smallest tau used for coupling strength G: the measured bound above plus a 0.05
    margin, interpolated linearly in G."""
    return float(np.interp(-G, TAU_STABLE_G, TAU_STABLE_MIN))


def batch_256(n: int = 256, seed: int = 4, steps: int = 2000, K: int = 100,
              storage: int = F16_OFFSET) -> List[Lattice]:
    rng = np.random.default_rng(1000 + seed)
    sides = rng.integers(1, 17, size=n) * 64
    Gs = rng.uniform(-6.0, -5.0, size=n)
    # tau uniform in [0.6, 1.2] restricted to the scheme's stable part for each G
    taus = np.array([rng.uniform(max(0.6, tau_min_stable(g)), 1.2) for g in Gs])
    rfrac = rng.uniform(0.1, 0.35, size=n)
    out = []
    for k in range(n):
        s = int(sides[k])
        out.append(Lattice(s, s, storage=storage, G=float(Gs[k]), tau=float(taus[k]),
                           droplets=[(s / 2.0, s / 2.0, float(rfrac[k] * s))],
                           seed=seed * 100000 + k, steps=steps, K=K, mlp=MLP_BF16,
                           weight_seed=10 + seed))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    job: Lattice


# Shan-Chen mechanical-stability coexistence densities of the scheme's equation of state
# p = rho/3 + G psi^2/6 with psi = 1 - exp(-rho): the vapour / liquid pair solving equal
# pressure and the integral condition (scipy quadrature and root finding, the routine the
# oracle's flat-interface pin checks the oracle against), tabulated every 0.1 in G.
COEX_G = (5.0, 5.1, 5.2, 5.3, 5.4, 5.5, 5.6, 5.7, 5.8, 5.9, 6.0)     # -G
COEX_VAPOUR = (0.1564, 0.1437, 0.1324, 0.1222, 0.1131, 0.1048, 0.0973, 0.0905, 0.0843, 0.0786, 0.0733)
COEX_LIQUID = (1.9324, 2.0111, 2.0877, 2.1625, 2.2357, 2.3075, 2.3780, 2.4473, 2.5155, 2.5827, 2.6490)


def coexistence(G: float) -> Tuple[float, float]:
    """(vapour, liquid) coexistence densities for G in [-6, -5], interpolated linearly."""
    return (float(np.interp(-G, COEX_G, COEX_VAPOUR)), float(np.interp(-G, COEX_G, COEX_LIQUID)))


def serve_tau(G: float) -> float:
    """Relaxation time of a served job: the paper's tau = 1 (Sec. III-A) up to G = -5.5,
    raised linearly to 1.2 at G = -6.  Served jobs hold up to eight large droplets that
    coalesce over up to 20000 steps.  In FP64 oracle runs at G = -5.9 started from 2.0 / 0.15,
    the flow reaches |u| = 0.6 and the field blows up within 1900 steps at tau = 1.16 (|u|
    stays near 0.65 even at tau = 1.3); started from the coexistence densities (below) at
    tau = 1.16, |u| stays below 0.26.  Served jobs therefore start at coexistence, with this
    tau."""
    return 1.0 + 0.4 * max(0.0, -G - 5.5)


def serve_poisson(n_requests: int = 500, rate_hz: float = 200.0, seed: int = 5,
                  side_max: int = 2048, steps_range=(1000, 20000), K: int = 100,
                  storage: int = F16_OFFSET) -> List[Request]:
    rng = np.random.default_rng(2000 + seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for k in range(n_requests):
        side = int(rng.integers(2, side_max // 32 + 1)) * 32
        nd = int(rng.integers(1, 9))
        cx = rng.uniform(0.0, side, size=nd)
        cy = rng.uniform(0.0, side, size=nd)
        r = rng.uniform(6.0, max(6.0, 0.3 * side), size=nd)
        G = float(rng.uniform(-6.0, -5.0))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        rho_v, rho_l = coexistence(G)
        job = Lattice(side, side, storage=storage, G=G, tau=serve_tau(G), rho_in=rho_l, rho_out=rho_v,
                      droplets=[(float(a), float(b), float(c)) for a, b, c in zip(cx, cy, r)],
                      seed=seed * 1000000 + k, steps=steps, K=K, mlp=MLP_BF16,
                      weight_seed=10 + seed)
        reqs.append(Request(float(t[k]), job))
    return reqs


def random_populations(nx: int, ny: int, seed: int, lo: float = 0.01, hi: float = 0.3) -> np.ndarray:
    """Arbitrary positive populations f[9, ny, nx] (for step-level parity on non-equilibrium input)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(9, ny, nx))


def sine_rho(nx: int, ny: int, a: float, b: float, axis: int = 0) -> np.ndarray:
    """Density field a + b sin(2 pi x / nx) (axis 0) or along y (axis 1).  Only a
    closed-form test input; the metrics computed from it live elsewhere."""
    if axis == 0:
        x = np.arange(nx)
        return np.broadcast_to(a + b * np.sin(2 * np.pi * x / nx), (ny, nx)).copy()
    y = np.arange(ny)
    return np.broadcast_to((a + b * np.sin(2 * np.pi * y / ny))[:, None], (ny, nx)).copy()

"""Seeded inputs for the "same state" parity tests (test infrastructure).

Every state handed to both sides comes from here: the oracle's own droplet initialisation
and steps (seeded), or a seeded draw, then made exactly representable in the lattice's
storage type, so that pl_set_state stores it without rounding and the oracle reads the very
values the GPU holds.  No state produced by the CUDA path ever feeds the oracle.

The FP16-offset exchange format written out here is the library's documented one: ten FP16
planes per buffer, the offsets h_0..h_8 and the reference densities r, with
f_i(x) = 2^-10 h_i(x) + Wr_i r(x - c_i), Wr = (1824, 456 x4, 114 x4) / 4096.
"""
import numpy as np

import oracle as O

F64, F32, F16 = 0, 1, 2

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WREF = np.array([1824, 456, 456, 456, 456, 114, 114, 114, 114], dtype=np.float64) / 4096.0
SCALE = 1024.0


def oracle_droplet_state(nx, ny, droplets, steps=0, G=-5.5, tau=1.0, seed=3, rho_in=2.0, rho_out=0.15):
    """FP64 populations f[9, ny, nx]: the oracle's initial droplet state advanced `steps`."""
    f = O.init_equilibrium(O.init_rho(nx, ny, droplets, rho_in, rho_out, 2.0, 0.01, seed))
    if steps:
        O.step(f, steps, G, tau)
    return f


def source_refs(r):
    """r(x - c_i) at every cell x, for each direction i: [9, ny, nx]."""
    return np.stack([np.roll(np.roll(r, CY[i], axis=0), CX[i], axis=1) for i in range(9)])


def f16(v):
    """Round to the nearest FP16 number, returned as FP64."""
    return v.astype(np.float16).astype(np.float64)


def encode_f16(f):
    """FP16-offset storage of populations f as pl_set_state writes it: r = fp16(rho) with rho
    summed in order 0..8 in FP64, h_i = fp16(2^10 (f_i - Wr_i r(x - c_i))), both rounded to
    nearest.  Returns (h[9, ny, nx], r[ny, nx]) as float16 arrays."""
    rho = f[0].copy()
    for i in range(1, 9):
        rho = rho + f[i]
    r = rho.astype(np.float16)
    h = ((f - WREF[:, None, None] * source_refs(r.astype(np.float64))) * SCALE).astype(np.float16)
    return h, r


def decode_f16(h, r):
    return h.astype(np.float64) / SCALE + WREF[:, None, None] * source_refs(r.astype(np.float64))


def stored(f, storage):
    """FP64 populations near f that the storage type holds exactly: storing them
    (pl_set_state) and reading them back (pl_get_state) returns them unchanged.  FP32: f
    rounded to nearest.  FP16-offset: the references r = fp16(rho(f)), the moving offsets
    rounded to nearest, and the rest offset chosen so that each cell's density is r within half
    an FP16 unit of h_0 - so the density of the result rounds to r again and encoding it
    reproduces the same offsets."""
    if storage == F64:
        return f.copy()
    if storage == F32:
        return f.astype(np.float32).astype(np.float64)
    _, r = encode_f16(f)
    r = r.astype(np.float64)
    rs = WREF[:, None, None] * source_refs(r)
    g = np.empty_like(f)
    g[1:] = f16((f[1:] - rs[1:]) * SCALE) / SCALE + rs[1:]
    g[0] = f16((r - rs[0] - g[1:].sum(axis=0)) * SCALE) / SCALE + rs[0]
    h2, r2 = encode_f16(g)
    assert np.array_equal(r2.astype(np.float64), r) and np.array_equal(decode_f16(h2, r2), g)
    return g


GRID = 2.0 ** -21


def exact_state(f, storage):
    """f moved onto a grid on which every per-cell sum the kernels form in FP32 is exact, so the
    density of a cell is the same number in FP32 on the GPU and in FP64 in the oracle:
      - FP32: values on multiples of 2^-21 (all below 4);
      - FP16-offset: references r on multiples of 2^-9 (FP16 numbers below 4, so Wr_i r is a
        multiple of 2^-21), moving offsets (2^-10 times FP16 numbers) on multiples of 2^-21,
        and the rest offset chosen so that each cell's density is r again (within one FP16
        rounding of 2^10 h_0 when |h_0| >= 2^-10), so that pl_set_state derives the same
        references;
      - FP64: unchanged."""
    if storage == F64:
        return f.copy()
    if storage == F32:
        return np.round(f / GRID) * GRID
    r = np.round(f.sum(axis=0) * 512.0) / 512.0
    assert r.min() > 0.0 and r.max() < 4.0
    rs = source_refs(r)
    h = np.zeros_like(f)
    for i in range(1, 9):
        hi = f16((f[i] - WREF[i] * rs[i]) * SCALE) / SCALE
        h[i] = np.round(hi / GRID) * GRID
    h0 = r - WREF[0] * r - (h[1:] + WREF[1:, None, None] * rs[1:]).sum(axis=0)
    h[0] = f16(h0 * SCALE) / SCALE
    assert np.array_equal(np.round(h[0] / GRID) * GRID, h[0])
    assert np.array_equal(f16(h * SCALE) / SCALE, h)
    out = h + WREF[:, None, None] * rs
    assert np.array_equal(encode_f16(out)[1].astype(np.float64), r)
    return out


def droplet_field_rho(nx, ny, droplets, rho_in, rho_out, width, noise_amp, seed):
    """A droplet density field of any size, quickly: tanh profiles (the shape of the set-up of
    Sec. III-A) evaluated only in each droplet's bounding box, the largest profile value per
    cell, plus uniform noise from numpy's PCG64.  A test input of the workload's structure
    (not the library's initialisation, whose noise comes from SplitMix64)."""
    phi = np.zeros((ny, nx))
    for cx, cy, r in droplets:
        ext = int(np.ceil(r + 20.0 * width)) + 1
        xs = np.arange(int(np.floor(cx)) - ext, int(np.floor(cx)) + ext + 1)
        ys = np.arange(int(np.floor(cy)) - ext, int(np.floor(cy)) + ext + 1)
        d = np.hypot(xs[None, :] - cx, ys[:, None] - cy)
        p = 0.5 * (1.0 - np.tanh((d - r) / width))
        iy, ix = np.ix_(ys % ny, xs % nx)
        if len(ys) > ny or len(xs) > nx:
            for a, yy in enumerate(ys % ny):
                phi[yy, xs % nx] = np.maximum(phi[yy, xs % nx], p[a])
        else:
            phi[iy, ix] = np.maximum(phi[iy, ix], p)
    rng = np.random.default_rng(seed)
    return rho_out + (rho_in - rho_out) * phi + noise_amp * (2.0 * rng.random((ny, nx)) - 1.0)


def at_rest(rho):
    """Populations of a fluid at rest, w_i rho (the lattice weights of Sec. II-A's D2Q9 reading)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w[:, None, None] * rho[None]

"""Seeded inputs for the "same state" parity tests (test infrastructure).

Every state handed to both sides comes from here: the oracle's own droplet initialisation
and steps (seeded), or a seeded draw, then made exactly representable in the lattice's
storage type, so that pl_set_state stores it without rounding and the oracle reads the very
values the GPU holds.  No state produced by the CUDA path ever feeds the oracle.
"""
import numpy as np

import oracle as O

F64, F32, F16 = 0, 1, 2


def oracle_droplet_state(nx, ny, droplets, steps=0, G=-5.5, tau=1.0, seed=3, rho_in=2.0, rho_out=0.15):
    """FP64 populations f[9, ny, nx]: the oracle's initial droplet state advanced `steps`."""
    f = O.init_equilibrium(O.init_rho(nx, ny, droplets, rho_in, rho_out, 2.0, 0.01, seed))
    if steps:
        O.step(f, steps, G, tau)
    return f


def stored(f, storage, rho_ref):
    """The FP64 values a storage type holds for populations f (round to nearest); FP16-offset
    encodes h = half(float(f) - float(w rho_ref)) and decodes float(h) + float(w rho_ref)."""
    if storage == F64:
        return f.copy()
    if storage == F32:
        return f.astype(np.float32).astype(np.float64)
    _, _, w = O.lattice_tables()
    off = (w * rho_ref).astype(np.float32)[:, None, None]
    h = (f.astype(np.float32) - off).astype(np.float16)
    return (h.astype(np.float32) + off).astype(np.float64)


EXACT_RHO_REF = 1.125          # w_i * 1.125 = 1/2, 1/8, 1/32: exact binary offsets
GRID = 2.0 ** -21


def exact_state(f, storage):
    """f moved onto a grid on which every per-cell sum the kernels form in FP32 is exact: values
    (FP32) or offsets from w_i * EXACT_RHO_REF (FP16-offset) that are multiples of 2^-21 with
    magnitudes below 4, so the density of a cell is the same number in FP32 on the GPU and in
    FP64 in the oracle.  FP64 storage is returned unchanged."""
    if storage == F64:
        return f.copy()
    if storage == F32:
        return np.round(f / GRID) * GRID
    _, _, w = O.lattice_tables()
    off = (w * EXACT_RHO_REF)[:, None, None]
    h = np.round((f - off) / GRID) * GRID
    h = h.astype(np.float16).astype(np.float64)       # FP16-representable, still on the grid
    h = np.round(h / GRID) * GRID
    return h + off

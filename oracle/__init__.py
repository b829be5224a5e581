"""FP64 CPU oracle of the PINN-LBM hot path — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

Thin ctypes marshalling over ``pinnlbm_oracle.c``; every number of the lattice,
the metrics, the network and the correction is computed there.  The network's
training (Eqs. 3-8) is the numpy module ``oracle.train``.  Arrays are numpy
float64 in the layout f[i, y, x] (direction-major, x fastest).
"""
import ctypes
import os

import numpy as np

from .build import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)

# Metric record fields returned by orc_metrics_rho (Eqs. 9-15).
METRIC_FIELDS = ("mass", "W", "G_max", "delta_rho", "W_eff", "E_int",
                 "rho_max", "rho_min", "sum_g", "sum_g2", "count")
LAPLACE_FIELDS = ("R_eq", "rho_in", "rho_out", "p_in", "p_out", "dP")


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        i, d, u64, vp = ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64, u64]
        L.orc_uniform01.restype = d
        L.orc_uniform01.argtypes = [u64, u64]
        L.orc_equilibrium.argtypes = [d, d, d, _dp]
        L.orc_psi.restype = d
        L.orc_psi.argtypes = [d, d]
        L.orc_pressure.restype = d
        L.orc_pressure.argtypes = [d, d, d]
        L.orc_density.argtypes = [i, i, _dp, _dp]
        L.orc_momentum.argtypes = [i, i, _dp, _dp, _dp]
        L.orc_sc_force.argtypes = [i, i, _dp, d, _dp, _dp]
        L.orc_collide.argtypes = [i, i, _dp, _dp, _dp, d, _dp]
        L.orc_stream.argtypes = [i, i, _dp, _dp]
        L.orc_step.restype = i
        L.orc_step.argtypes = [i, i, _dp, i, d, d, d]
        L.orc_init_rho.argtypes = [i, i, i, _dp, _dp, _dp, d, d, d, d, u64, _dp]
        L.orc_init_equilibrium.argtypes = [i, i, _dp, _dp]
        L.orc_grad_mag.argtypes = [i, i, _dp, _dp]
        L.orc_metrics_rho.argtypes = [i, i, _dp, d, _dp]
        L.orc_laplace.argtypes = [i, i, _dp, d, d, d, d, d, _dp]
        L.orc_mlp_blob_size.restype = ctypes.c_long
        L.orc_round_bf16.restype = d
        L.orc_round_bf16.argtypes = [d]
        L.orc_mlp_forward.argtypes = [_fp, i, d, d, _dp]
        L.orc_mlp_field.argtypes = [i, i, _fp, i, _dp]
        L.orc_correct.restype = i
        L.orc_correct.argtypes = [i, i, _dp, _fp, i, vp, d, d, d]
        L.orc_mass.restype = d
        L.orc_mass.argtypes = [i, i, _dp]
        L.orc_run.restype = i
        L.orc_run.argtypes = [i, i, _dp, i, ctypes.c_long, i, d, d, d, _fp, i, d, d, d]
        L.orc_mlp_blob_size_n.restype = ctypes.c_long
        L.orc_mlp_blob_size_n.argtypes = [i]
        L.orc_mlp_forward_n.argtypes = [_fp, i, i, _dp, _dp]
        L.orc_mlp_field_n.argtypes = [i, i, _fp, i, i, vp, _dp]
        L.orc_correct_n.restype = i
        L.orc_correct_n.argtypes = [i, i, _dp, _fp, i, i, vp, d, d, d]
        L.orc_correct_eps.restype = i
        L.orc_correct_eps.argtypes = [i, i, _dp, _fp, i, i, vp, d, d, d, d]
        L.orc_run_eps.restype = i
        L.orc_run_eps.argtypes = [i, i, _dp, i, ctypes.c_long, i, d, d, d, _fp, i, i, d, d, d, d]
        L.orc_run_n.restype = i
        L.orc_run_n.argtypes = [i, i, _dp, i, ctypes.c_long, i, d, d, d, _fp, i, i, d, d, d]
        L.orc_mlp_init_weights.argtypes = [i, u64, _fp]
        L.orc_num_threads.restype = i
        L.orc_set_num_threads.argtypes = [i]
        L.orc_lattice_tables.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
        _lib = L
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f(a):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_fp)


# ----------------------------------------------------------------------------- tables / helpers

def lattice_tables():
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    lib().orc_lattice_tables(cx, cy, w)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:])


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    lib().orc_set_num_threads(int(n))


def splitmix64(seed, k):
    return lib().orc_splitmix64(seed & (2**64 - 1), k & (2**64 - 1))


def uniform01(seed, k):
    return lib().orc_uniform01(seed & (2**64 - 1), k)


def equilibrium(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_equilibrium(rho, ux, uy, _d(out))
    return out


def psi(rho, rho0=1.0):
    return lib().orc_psi(rho, rho0)


def pressure(rho, G, rho0=1.0):
    return lib().orc_pressure(rho, G, rho0)


def round_bf16(v):
    return lib().orc_round_bf16(float(v))


# ----------------------------------------------------------------------------- field operations

def density(f):
    _, ny, nx = f.shape
    rho = np.zeros((ny, nx))
    lib().orc_density(nx, ny, _d(f), _d(rho))
    return rho


def momentum(f):
    _, ny, nx = f.shape
    jx, jy = np.zeros((ny, nx)), np.zeros((ny, nx))
    lib().orc_momentum(nx, ny, _d(f), _d(jx), _d(jy))
    return jx, jy


def sc_force(psi_field, G):
    ny, nx = psi_field.shape
    Fx, Fy = np.zeros((ny, nx)), np.zeros((ny, nx))
    lib().orc_sc_force(nx, ny, _d(np.ascontiguousarray(psi_field, dtype=np.float64)), G, _d(Fx), _d(Fy))
    return Fx, Fy


def collide(f, Fx, Fy, tau):
    _, ny, nx = f.shape
    out = np.zeros_like(f)
    lib().orc_collide(nx, ny, _d(f), _d(np.ascontiguousarray(Fx)), _d(np.ascontiguousarray(Fy)), tau, _d(out))
    return out


def stream(fpost):
    _, ny, nx = fpost.shape
    out = np.zeros_like(fpost)
    lib().orc_stream(nx, ny, _d(np.ascontiguousarray(fpost)), _d(out))
    return out


def step(f, n, G, tau, rho0=1.0):
    """Advance f (modified in place) by n steps of Eq. 1."""
    _, ny, nx = f.shape
    st = lib().orc_step(nx, ny, _d(f), int(n), G, tau, rho0)
    if st != 0:
        raise MemoryError("oracle step: allocation failed")
    return f


def init_rho(nx, ny, droplets, rho_in, rho_out, width, noise_amp, seed):
    d = np.asarray(droplets, dtype=np.float64).reshape(-1, 3)
    cx, cy, r = (np.ascontiguousarray(d[:, k]) for k in range(3))
    rho = np.zeros((ny, nx))
    lib().orc_init_rho(nx, ny, len(d), _d(cx), _d(cy), _d(r), rho_in, rho_out, width, noise_amp,
                       seed & (2**64 - 1), _d(rho))
    return rho


def init_equilibrium(rho):
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    lib().orc_init_equilibrium(nx, ny, _d(np.ascontiguousarray(rho, dtype=np.float64)), _d(f))
    return f


def grad_mag(rho):
    ny, nx = rho.shape
    g = np.zeros((ny, nx))
    lib().orc_grad_mag(nx, ny, _d(np.ascontiguousarray(rho, dtype=np.float64)), _d(g))
    return g


def metrics_rho(rho, threshold=0.01):
    ny, nx = rho.shape
    out = np.zeros(len(METRIC_FIELDS))
    lib().orc_metrics_rho(nx, ny, _d(np.ascontiguousarray(rho, dtype=np.float64)), threshold, _d(out))
    m = dict(zip(METRIC_FIELDS, out.tolist()))
    m["count"] = int(round(m["count"]))
    return m


def laplace(rho, cx, cy, width, G, rho0=1.0):
    ny, nx = rho.shape
    out = np.zeros(len(LAPLACE_FIELDS))
    lib().orc_laplace(nx, ny, _d(np.ascontiguousarray(rho, dtype=np.float64)), cx, cy, width, G, rho0, _d(out))
    return dict(zip(LAPLACE_FIELDS, out.tolist()))


def mass(f):
    _, ny, nx = f.shape
    return lib().orc_mass(nx, ny, _d(f))


# ----------------------------------------------------------------------------- network / correction

MLP_F64 = 0
MLP_BF16 = 1


def mlp_blob_size(n_in=2):
    """Weight blob length for n_in network inputs (2: the paper's (x^, y^); 11: with the
    density stencil)."""
    return lib().orc_mlp_blob_size_n(int(n_in))


def mlp_init_weights(seed, n_in=2):
    """The seeded FP32 weight blob (fan-in uniform from SplitMix64, counter = blob index)."""
    out = np.zeros(mlp_blob_size(n_in), dtype=np.float32)
    lib().orc_mlp_init_weights(int(n_in), seed & (2**64 - 1), _f(out))
    return out


def mlp_forward(blob, xh, yh, mode=MLP_F64):
    out = np.zeros(3)
    lib().orc_mlp_forward(_f(np.ascontiguousarray(blob, dtype=np.float32)), mode, xh, yh, _d(out))
    return out


def mlp_forward_n(blob, inputs, mode=MLP_F64):
    """Network on an explicit input vector (2 or 11 values)."""
    x = np.ascontiguousarray(inputs, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_mlp_forward_n(_f(np.ascontiguousarray(blob, dtype=np.float32)), mode, int(x.size), _d(x), _d(out))
    return out


def mlp_field(blob, nx, ny, mode=MLP_F64, n_in=2, rho=None):
    """Network outputs on every cell, (3, ny, nx); n_in = 11 reads the density field rho."""
    out = np.zeros((3, ny, nx))
    r = None
    if n_in == 11:
        r = np.ascontiguousarray(rho, dtype=np.float64)
        assert r.shape == (ny, nx)
    lib().orc_mlp_field_n(nx, ny, _f(np.ascontiguousarray(blob, dtype=np.float32)), mode, int(n_in),
                          None if r is None else r.ctypes.data, _d(out))
    return out


def correct(f, blob, beta_rho, beta_u, M0, mode=MLP_F64, mlp_out=None, n_in=2, eps=0.0):
    """Apply the interface correction to f in place; returns the status (0 or -4).  Cells whose
    mask g / G_max is not above eps are outside the interface band (mask 0)."""
    _, ny, nx = f.shape
    b = np.ascontiguousarray(blob, dtype=np.float32)
    out3 = None
    if mlp_out is not None:
        out3 = np.ascontiguousarray(mlp_out, dtype=np.float64)
    return lib().orc_correct_eps(nx, ny, _d(f), _f(b), mode, int(n_in), None if out3 is None else out3.ctypes.data,
                                 beta_rho, beta_u, M0, float(eps))


def run(f, nsteps, G, tau, rho0=1.0, K=0, blob=None, mode=MLP_F64, beta_rho=0.1, beta_u=0.01,
        M0=None, step0=0, n_in=2, eps=0.0):
    """Coupled run (Sec. II-C): nsteps of Eq. 1, correction after every K-th step (interface
    band of the correction: mask above eps)."""
    _, ny, nx = f.shape
    if M0 is None:
        M0 = mass(f)
    b = None if blob is None else np.ascontiguousarray(blob, dtype=np.float32)
    return lib().orc_run_eps(nx, ny, _d(f), int(nsteps), int(step0), int(K), G, tau, rho0,
                             None if b is None else _f(b), mode, int(n_in), beta_rho, beta_u, M0, float(eps))

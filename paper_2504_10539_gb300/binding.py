"""ctypes binding of ``libpinnlbm.so`` (C ABI in include/pinnlbm.h).

Argument marshalling only: each ``pl_*`` function here calls the C function of
the same name and raises :class:`PLError` on a non-zero status.  Every step of
the hot path runs in the library's CUDA kernels; if the library has not been
built this module raises instead of computing anything another way.

``Lattice`` is a convenience owner: it allocates the caller-side device buffer
with torch (device memory and streams are the only things torch provides) and
keeps the handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpinnlbm.so")

PL_OK = 0
PL_ERR_INVALID_ARG = -1
PL_ERR_CUDA = -2
PL_ERR_BUDGET = -3
PL_ERR_NONPHYSICAL = -4
PL_ERR_TIMEOUT = -5
PL_ERR_STATE = -6

PL_F64, PL_F32, PL_F16_OFFSET = 0, 1, 2
PL_TRAIN_SIMT, PL_TRAIN_TC = 0, 1
PL_MLP_F64, PL_MLP_F32, PL_MLP_BF16 = 0, 1, 2
PL_MAX_DROPLETS = 4096


class pl_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("mlp", ctypes.c_int32), ("G", ctypes.c_double), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("mask_eps", ctypes.c_double), ("beta_rho", ctypes.c_double),
                ("beta_u", ctypes.c_double), ("threshold", ctypes.c_double), ("mlp_in", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class pl_droplet(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double)]


class pl_metric_record(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("W", ctypes.c_double), ("G_max", ctypes.c_double),
                ("delta_rho", ctypes.c_double), ("W_eff", ctypes.c_double), ("E_int", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("rho_min", ctypes.c_double), ("sum_g", ctypes.c_double),
                ("sum_g2", ctypes.c_double), ("count", ctypes.c_int64), ("R_eq", ctypes.c_double),
                ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double), ("p_in", ctypes.c_double),
                ("p_out", ctypes.c_double), ("dP", ctypes.c_double), ("mass0", ctypes.c_double),
                ("step", ctypes.c_int64), ("status", ctypes.c_int32), ("corrections", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pl_job_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("steps", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32), ("metrics", pl_metric_record)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "metrics")}
        d["metrics"] = self.metrics.as_dict()
        return d


class pl_train_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("lambda_phys", ctypes.c_double), ("lambda_int", ctypes.c_double),
                ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class PLError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = "%s failed: %s (%d)" % (fn, pl_status_string(status), status)
        if status == PL_ERR_CUDA:
            msg += ", cudaError %d" % _L().pl_last_cuda_error()
        super().__init__(msg)


_lib = None


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpinnlbm.so is not built (expected at %s); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, d, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                    ctypes.c_double, ctypes.c_size_t)
        P = ctypes.POINTER
        sigs = {
            "pl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "pl_last_cuda_error": (ctypes.c_int, []),
            "pl_kernel_launches": (ctypes.c_int, [P(i64)]),
            "pl_params_default": (ctypes.c_int, [P(pl_params), i32, i32]),
            "pl_lattice_bytes": (ctypes.c_int, [P(pl_params), P(sz)]),
            "pl_lattice_create": (ctypes.c_int, [P(pl_params), vp, sz, vp, P(vp)]),
            "pl_lattice_init_droplets": (ctypes.c_int, [vp, P(pl_droplet), ctypes.c_int, d, d, d, d, u64]),
            "pl_lattice_init_rho": (ctypes.c_int, [vp, P(d)]),
            "pl_mlp_blob_size": (ctypes.c_int, []),
            "pl_mlp_blob_size_for": (ctypes.c_int, [ctypes.c_int32]),
            "pl_set_mlp_weights": (ctypes.c_int, [vp, P(ctypes.c_float), sz]),
            "pl_init_mlp_weights": (ctypes.c_int, [vp, u64]),
            "pl_batch_init_mlp_weights": (ctypes.c_int, [vp, i32, u64]),
            "pl_step": (ctypes.c_int, [vp, i32]),
            "pl_apply_correction": (ctypes.c_int, [vp]),
            "pl_run": (ctypes.c_int, [vp, i32, i32]),
            "pl_metrics": (ctypes.c_int, [vp, P(pl_metric_record)]),
            "pl_get_rho": (ctypes.c_int, [vp, P(d)]),
            "pl_get_mlp_field": (ctypes.c_int, [vp, P(d)]),
            "pl_get_state": (ctypes.c_int, [vp, P(d), P(i64)]),
            "pl_set_state": (ctypes.c_int, [vp, P(d), i64]),
            "pl_lattice_status": (ctypes.c_int, [vp]),
            "pl_metrics_noalloc": (ctypes.c_int, [vp, i32, i32, i32, i32, d, d, vp, P(pl_metric_record)]),
            "pl_batch_overhead_bytes": (ctypes.c_int, [i32, P(sz)]),
            "pl_batch_job_bytes": (ctypes.c_int, [P(pl_params), P(sz)]),
            "pl_batch_create": (ctypes.c_int, [i32, i32, i32, i32, vp, sz, vp, P(vp)]),
            "pl_batch_set_mlp_weights": (ctypes.c_int, [vp, P(ctypes.c_float), sz]),
            "pl_batch_submit": (ctypes.c_int, [vp, P(pl_params), P(pl_droplet), ctypes.c_int, d, d, d, d, u64, i64,
                                               P(i64)]),
            "pl_batch_advance": (ctypes.c_int, [vp, i32]),
            "pl_batch_poll": (ctypes.c_int, [vp, P(pl_job_result), i32, P(i32)]),
            "pl_batch_info": (ctypes.c_int, [vp, P(i32), P(i64), P(sz), P(sz)]),
            "pl_batch_get_state": (ctypes.c_int, [vp, i64, P(d), P(i64)]),
            "pl_batch_autotune": (ctypes.c_int, [vp, i32, P(i32)]),
            "pl_batch_metrics": (ctypes.c_int, [vp, P(pl_job_result), i32, P(i32)]),
            "pl_batch_interval_times": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float)]),
            "pl_batch_destroy": (ctypes.c_int, [vp]),
            "pl_destroy": (ctypes.c_int, [vp]),
            "pl_selftest_wait_timeout": (ctypes.c_int, [vp, i64, vp]),
            "pl_get_mlp_weights": (ctypes.c_int, [vp, P(ctypes.c_float), sz]),
            "pl_train_params_default": (ctypes.c_int, [P(pl_train_params)]),
            "pl_trainer_bytes": (ctypes.c_int, [P(pl_params), i32, P(sz)]),
            "pl_trainer_create": (ctypes.c_int, [vp, P(pl_train_params), i32, vp, sz, P(vp)]),
            "pl_train": (ctypes.c_int, [vp, i32]),
            "pl_train_losses": (ctypes.c_int, [vp, P(d), i32]),
            "pl_train_gradient": (ctypes.c_int, [vp, P(d), P(d)]),
            "pl_run_trained": (ctypes.c_int, [vp, i32, i32, i32]),
            "pl_trainer_destroy": (ctypes.c_int, [vp]),
        }
        for name, (res, args) in sigs.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
    return _lib


def lib():
    return _L()


def _chk(fn, st):
    if st != PL_OK:
        raise PLError(fn, st)
    return st


def _dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------- C ABI, one wrapper per call

def pl_status_string(status: int) -> str:
    return _L().pl_status_string(status).decode()


def pl_last_cuda_error() -> int:
    return _L().pl_last_cuda_error()


def pl_kernel_launches() -> int:
    n = ctypes.c_int64()
    _chk("pl_kernel_launches", _L().pl_kernel_launches(ctypes.byref(n)))
    return n.value


def pl_params_default(nx: int, ny: int, **kw) -> pl_params:
    p = pl_params()
    _chk("pl_params_default", _L().pl_params_default(ctypes.byref(p), nx, ny))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def pl_lattice_bytes(p: pl_params) -> int:
    n = ctypes.c_size_t()
    _chk("pl_lattice_bytes", _L().pl_lattice_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def pl_lattice_create(p: pl_params, dev_ptr: int, nbytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    _chk("pl_lattice_create", _L().pl_lattice_create(ctypes.byref(p), ctypes.c_void_p(dev_ptr), nbytes,
                                                      ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def pl_lattice_init_droplets(h, droplets: Sequence, rho_in, rho_out, width, noise_amp, seed):
    n = len(droplets)
    arr = (pl_droplet * max(n, 1))(*[pl_droplet(*map(float, d)) for d in droplets])
    return _chk("pl_lattice_init_droplets", _L().pl_lattice_init_droplets(
        ctypes.c_void_p(h), arr, n, rho_in, rho_out, width, noise_amp, seed & (2 ** 64 - 1)))


def pl_lattice_init_rho(h, rho: np.ndarray):
    r = np.ascontiguousarray(rho, dtype=np.float64)
    return _chk("pl_lattice_init_rho", _L().pl_lattice_init_rho(ctypes.c_void_p(h), _dptr(r)))


def pl_mlp_blob_size() -> int:
    return _L().pl_mlp_blob_size()


def pl_mlp_blob_size_for(mlp_in: int) -> int:
    n = _L().pl_mlp_blob_size_for(mlp_in)
    _chk("pl_mlp_blob_size_for", min(n, 0))
    return n


def pl_set_mlp_weights(h, blob: np.ndarray):
    b = np.ascontiguousarray(blob, dtype=np.float32)
    return _chk("pl_set_mlp_weights", _L().pl_set_mlp_weights(
        ctypes.c_void_p(h), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), b.size))


def pl_init_mlp_weights(h, seed: int):
    return _chk("pl_init_mlp_weights", _L().pl_init_mlp_weights(ctypes.c_void_p(h), seed & (2 ** 64 - 1)))


def pl_step(h, n: int):
    return _chk("pl_step", _L().pl_step(ctypes.c_void_p(h), n))


def pl_apply_correction(h):
    return _chk("pl_apply_correction", _L().pl_apply_correction(ctypes.c_void_p(h)))


def pl_run(h, nsteps: int, K: int):
    return _chk("pl_run", _L().pl_run(ctypes.c_void_p(h), nsteps, K))


def pl_metrics(h) -> dict:
    m = pl_metric_record()
    _chk("pl_metrics", _L().pl_metrics(ctypes.c_void_p(h), ctypes.byref(m)))
    return m.as_dict()


def pl_get_rho(h, nx: int, ny: int) -> np.ndarray:
    out = np.empty((ny, nx), dtype=np.float64)
    _chk("pl_get_rho", _L().pl_get_rho(ctypes.c_void_p(h), _dptr(out)))
    return out


def pl_get_mlp_field(h, nx: int, ny: int) -> np.ndarray:
    out = np.empty((3, ny, nx), dtype=np.float64)
    _chk("pl_get_mlp_field", _L().pl_get_mlp_field(ctypes.c_void_p(h), _dptr(out)))
    return out


def pl_get_state(h, nx: int, ny: int):
    out = np.empty((9, ny, nx), dtype=np.float64)
    step = ctypes.c_int64()
    _chk("pl_get_state", _L().pl_get_state(ctypes.c_void_p(h), _dptr(out), ctypes.byref(step)))
    return out, step.value


def pl_set_state(h, f: np.ndarray, step: int = 0):
    a = np.ascontiguousarray(f, dtype=np.float64)
    return _chk("pl_set_state", _L().pl_set_state(ctypes.c_void_p(h), _dptr(a), step))


def pl_lattice_status(h) -> int:
    return _L().pl_lattice_status(ctypes.c_void_p(h))


def pl_metrics_noalloc(dev_ptr: int, nx: int, ny: int, pitch: int, storage: int, rho_ref: float,
                       threshold: float, stream: int) -> dict:
    """Metrics of caller-held populations without any device allocation (static scratch)."""
    m = pl_metric_record()
    _chk("pl_metrics_noalloc", _L().pl_metrics_noalloc(ctypes.c_void_p(dev_ptr), nx, ny, pitch, storage, rho_ref,
                                                        threshold, ctypes.c_void_p(stream), ctypes.byref(m)))
    return m.as_dict()


def pl_destroy(h):
    return _chk("pl_destroy", _L().pl_destroy(ctypes.c_void_p(h)))


def pl_selftest_wait_timeout(dev_status_ptr: int, limit_ns: int, stream: int = 0) -> int:
    """Runs the bounded-wait self-test; returns the status it reports (PL_ERR_TIMEOUT expected)."""
    return _L().pl_selftest_wait_timeout(ctypes.c_void_p(dev_status_ptr), int(limit_ns), ctypes.c_void_p(stream))


def pl_get_mlp_weights(h, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float32)
    _chk("pl_get_mlp_weights", _L().pl_get_mlp_weights(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n))
    return out


def pl_train_params_default(**kw) -> pl_train_params:
    tp = pl_train_params()
    _chk("pl_train_params_default", _L().pl_train_params_default(ctypes.byref(tp)))
    for k, v in kw.items():
        setattr(tp, k, v)
    return tp


def pl_trainer_bytes(p: pl_params, max_epochs: int) -> int:
    out = ctypes.c_size_t(0)
    _chk("pl_trainer_bytes", _L().pl_trainer_bytes(ctypes.byref(p), int(max_epochs), ctypes.byref(out)))
    return out.value


def pl_trainer_create(lat_h, tp: pl_train_params, max_epochs: int, dev_ptr: int, nbytes: int) -> int:
    h = ctypes.c_void_p()
    _chk("pl_trainer_create", _L().pl_trainer_create(lat_h, ctypes.byref(tp), int(max_epochs), ctypes.c_void_p(dev_ptr),
                                                     nbytes, ctypes.byref(h)))
    return h.value


def pl_train(h, epochs: int):
    _chk("pl_train", _L().pl_train(h, int(epochs)))


def pl_train_losses(h, epochs: int) -> np.ndarray:
    out = np.zeros((epochs, 4))
    _chk("pl_train_losses", _L().pl_train_losses(h, _dptr(out), int(epochs)))
    return out


def pl_train_gradient(h, n: int):
    g, loss = np.zeros(n), np.zeros(4)
    _chk("pl_train_gradient", _L().pl_train_gradient(h, _dptr(g), _dptr(loss)))
    return g, loss


def pl_run_trained(h, nsteps: int, K: int, epochs: int):
    _chk("pl_run_trained", _L().pl_run_trained(h, int(nsteps), int(K), int(epochs)))


def pl_trainer_destroy(h):
    _chk("pl_trainer_destroy", _L().pl_trainer_destroy(h))


# ----------------------------------------------------------------------------- owner of one lattice

class Lattice:
    """One lattice over a torch-allocated device buffer, enqueuing on a torch stream."""

    def __init__(self, params: pl_params, device: str = "cuda", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.nbytes = pl_lattice_bytes(params)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        # a stream of its own (capturable into CUDA graphs, unlike the legacy default stream);
        # the buffer's allocation is ordered before any work on it
        self.stream = stream if stream is not None else torch.cuda.Stream(self.mem.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.mem.device))
        self.h = pl_lattice_create(params, self.mem.data_ptr(), self.nbytes, self.stream.cuda_stream)

    @classmethod
    def from_workload(cls, job, device="cuda", stream=None):
        """Build, initialise and load weights for a ``workloads.Lattice`` description."""
        lat = cls(job_params(job), device=device, stream=stream)
        lat.init_droplets(job.droplets, job.rho_in, job.rho_out, job.width, job.noise_amp, job.seed)
        if job.K > 0:
            lat.set_weights(job.weights())
        return lat

    def init_droplets(self, droplets, rho_in, rho_out, width, noise_amp, seed):
        pl_lattice_init_droplets(self.h, droplets, rho_in, rho_out, width, noise_amp, seed)

    def init_rho(self, rho):
        pl_lattice_init_rho(self.h, rho)

    def set_weights(self, blob):
        pl_set_mlp_weights(self.h, blob)

    def init_weights(self, seed):
        pl_init_mlp_weights(self.h, seed)

    def step(self, n):
        pl_step(self.h, n)

    def correct(self):
        pl_apply_correction(self.h)

    def run(self, nsteps, K):
        pl_run(self.h, nsteps, K)

    def metrics(self):
        return pl_metrics(self.h)

    def rho(self):
        return pl_get_rho(self.h, self.nx, self.ny)

    def mlp_field(self):
        return pl_get_mlp_field(self.h, self.nx, self.ny)

    def state(self):
        return pl_get_state(self.h, self.nx, self.ny)

    def set_state(self, f, step=0):
        pl_set_state(self.h, f, step)

    def status(self):
        return pl_lattice_status(self.h)

    def weights(self):
        return pl_get_mlp_weights(self.h, pl_mlp_blob_size_for(self.params.mlp_in))

    def close(self):
        if getattr(self, "h", None):
            pl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trainer:
    """Network training on a Lattice's state (Eqs. 3-8) over a torch-allocated device buffer;
    enqueues on the lattice's stream.  Keeps a reference to the lattice, so the lattice
    outlives it."""

    def __init__(self, lattice: Lattice, max_epochs: int = 300, **hyper):
        import torch
        self.lattice = lattice
        self.tp = pl_train_params_default(**hyper)
        self.max_epochs = max_epochs
        self.nbytes = pl_trainer_bytes(lattice.params, max_epochs)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=lattice.mem.device)
        lattice.stream.wait_stream(torch.cuda.current_stream(self.mem.device))
        self.h = pl_trainer_create(lattice.h, self.tp, max_epochs, self.mem.data_ptr(), self.nbytes)

    def train(self, epochs):
        pl_train(self.h, epochs)

    def losses(self, epochs):
        return pl_train_losses(self.h, epochs)

    def gradient(self):
        return pl_train_gradient(self.h, pl_mlp_blob_size())

    def run(self, nsteps, K, epochs):
        pl_run_trained(self.h, nsteps, K, epochs)

    def close(self):
        if getattr(self, "h", None):
            pl_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- batches of lattices

def pl_batch_overhead_bytes(max_jobs: int) -> int:
    n = ctypes.c_size_t()
    _chk("pl_batch_overhead_bytes", _L().pl_batch_overhead_bytes(max_jobs, ctypes.byref(n)))
    return n.value


def pl_batch_job_bytes(p: pl_params) -> int:
    n = ctypes.c_size_t()
    _chk("pl_batch_job_bytes", _L().pl_batch_job_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def pl_batch_create(storage: int, mlp: int, K: int, max_jobs: int, dev_ptr: int, nbytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    _chk("pl_batch_create", _L().pl_batch_create(storage, mlp, K, max_jobs, ctypes.c_void_p(dev_ptr), nbytes,
                                                  ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def pl_batch_set_mlp_weights(h, blob: np.ndarray):
    b = np.ascontiguousarray(blob, dtype=np.float32)
    return _chk("pl_batch_set_mlp_weights", _L().pl_batch_set_mlp_weights(
        ctypes.c_void_p(h), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), b.size))


def pl_batch_init_mlp_weights(h, mlp_in: int, seed: int):
    return _chk("pl_batch_init_mlp_weights", _L().pl_batch_init_mlp_weights(ctypes.c_void_p(h), mlp_in,
                                                                            seed & (2 ** 64 - 1)))


def pl_batch_submit(h, p: pl_params, droplets, rho_in, rho_out, width, noise_amp, seed, steps):
    """Returns the job id, or None when the batch has no room for it now (PL_ERR_BUDGET)."""
    n = len(droplets)
    arr = (pl_droplet * max(n, 1))(*[pl_droplet(*map(float, dd)) for dd in droplets])
    jid = ctypes.c_int64()
    st = _L().pl_batch_submit(ctypes.c_void_p(h), ctypes.byref(p), arr, n, rho_in, rho_out, width, noise_amp,
                              seed & (2 ** 64 - 1), steps, ctypes.byref(jid))
    if st == PL_ERR_BUDGET:
        return None
    _chk("pl_batch_submit", st)
    return jid.value


def pl_batch_advance(h, intervals: int = 1):
    return _chk("pl_batch_advance", _L().pl_batch_advance(ctypes.c_void_p(h), intervals))


def pl_batch_poll(h, max_results: int = 1024):
    out = (pl_job_result * max(max_results, 1))()
    n = ctypes.c_int32()
    _chk("pl_batch_poll", _L().pl_batch_poll(ctypes.c_void_p(h), out, max_results, ctypes.byref(n)))
    return [out[k].as_dict() for k in range(n.value)]


def pl_batch_info(h) -> dict:
    a, c, u, t = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_size_t()
    _chk("pl_batch_info", _L().pl_batch_info(ctypes.c_void_p(h), ctypes.byref(a), ctypes.byref(c), ctypes.byref(u),
                                              ctypes.byref(t)))
    return {"active": a.value, "cells": c.value, "arena_used": u.value, "arena_total": t.value}


def pl_batch_get_state(h, job_id: int, nx: int, ny: int):
    out = np.empty((9, ny, nx), dtype=np.float64)
    step = ctypes.c_int64()
    _chk("pl_batch_get_state", _L().pl_batch_get_state(ctypes.c_void_p(h), job_id, _dptr(out), ctypes.byref(step)))
    return out, step.value


def pl_batch_autotune(h, force: bool = False) -> int:
    r = ctypes.c_int32()
    _chk("pl_batch_autotune", _L().pl_batch_autotune(ctypes.c_void_p(h), int(force), ctypes.byref(r)))
    return r.value


def pl_batch_metrics(h, max_results: int = 4096):
    out = (pl_job_result * max(max_results, 1))()
    n = ctypes.c_int32()
    _chk("pl_batch_metrics", _L().pl_batch_metrics(ctypes.c_void_p(h), out, max_results, ctypes.byref(n)))
    return [out[k].as_dict() for k in range(n.value)]


def pl_batch_interval_times(h):
    s, t = ctypes.c_float(), ctypes.c_float()
    _chk("pl_batch_interval_times", _L().pl_batch_interval_times(ctypes.c_void_p(h), ctypes.byref(s),
                                                                  ctypes.byref(t)))
    return s.value, t.value


def pl_batch_destroy(h):
    return _chk("pl_batch_destroy", _L().pl_batch_destroy(ctypes.c_void_p(h)))


def job_params(job) -> pl_params:
    """C parameters of a ``workloads.Lattice`` description."""
    return pl_params_default(job.nx, job.ny, storage=job.storage, mlp=job.mlp, G=job.G, tau=job.tau, rho0=job.rho0,
                             mask_eps=getattr(job, "mask_eps", 0.0), beta_rho=job.beta_rho, beta_u=job.beta_u,
                             mlp_in=getattr(job, "mlp_in", 2))


class Batch:
    """A batch over a torch-allocated device buffer of `budget_bytes` (the device budget)."""

    def __init__(self, storage: int, mlp: int, K: int, budget_bytes: int, max_jobs: int = 1024, device="cuda",
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.mem = torch.empty(int(budget_bytes), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.mem.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.mem.device))
        self.K = K
        self.h = pl_batch_create(storage, mlp, K, max_jobs, self.mem.data_ptr(), int(budget_bytes),
                                 self.stream.cuda_stream)
        self.jobs = {}

    def set_weights(self, blob):
        pl_batch_set_mlp_weights(self.h, blob)

    def init_weights(self, seed, mlp_in=2):
        pl_batch_init_mlp_weights(self.h, mlp_in, seed)

    def submit(self, job, steps=None):
        jid = pl_batch_submit(self.h, job_params(job), job.droplets, job.rho_in, job.rho_out, job.width,
                              job.noise_amp, job.seed, int(steps if steps is not None else job.steps))
        if jid is not None:
            self.jobs[jid] = job
        return jid

    def advance(self, intervals=1):
        pl_batch_advance(self.h, intervals)

    def job_bytes(self, job) -> int:
        """Arena bytes the job's lattice takes (pl_batch_job_bytes)."""
        return pl_batch_job_bytes(job_params(job))

    def arena_bytes(self) -> int:
        """Size of the arena the jobs are carved from (the budget minus the batch's head)."""
        return pl_batch_info(self.h)["arena_total"]

    def poll(self):
        return pl_batch_poll(self.h)

    def info(self):
        return pl_batch_info(self.h)

    def state(self, jid):
        job = self.jobs[jid]
        return pl_batch_get_state(self.h, jid, job.nx, job.ny)

    def autotune(self, force=False):
        return pl_batch_autotune(self.h, force)

    def close(self):
        if getattr(self, "h", None):
            pl_batch_destroy(self.h)
            self.h = None
        self.mem = None             # the device buffer goes with the handle

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

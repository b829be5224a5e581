"""C-ABI checks that need no GPU: the library loads, exports every function the
header declares, and the host-only calls behave as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2504_10539_gb300 import binding as B
from paper_2504_10539_gb300 import build as pkg_build
from paper_2504_10539_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return B.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^PL_API\s+[\w\s\*]+?\b(pl_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pl_lattice_bytes", "pl_lattice_create", "pl_lattice_init_droplets", "pl_step",
                 "pl_apply_correction", "pl_metrics", "pl_destroy", "pl_run", "pl_set_mlp_weights"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for st in (B.PL_OK, B.PL_ERR_INVALID_ARG, B.PL_ERR_CUDA, B.PL_ERR_BUDGET, B.PL_ERR_NONPHYSICAL,
               B.PL_ERR_TIMEOUT, B.PL_ERR_STATE):
        assert B.pl_status_string(st) != "unknown status"
    assert B.pl_status_string(12345) == "unknown status"


def test_blob_size_agrees_everywhere(lib):
    assert B.pl_mlp_blob_size() == wl.mlp_blob_size() == O.mlp_blob_size() == 33475


def test_params_default_and_bytes(lib):
    p = B.pl_params_default(64, 48)
    assert (p.nx, p.ny, p.storage, p.mlp) == (64, 48, B.PL_F32, B.PL_MLP_BF16)
    assert p.G == -5.5 and p.tau == 1.0 and p.threshold == 0.01
    n32 = B.pl_lattice_bytes(p)
    assert n32 >= 2 * 9 * 64 * 48 * 4
    p.storage = B.PL_F16_OFFSET
    n16 = B.pl_lattice_bytes(p)
    assert 2 * 9 * 64 * 48 * 2 <= n16 < n32
    p.storage, p.mlp = B.PL_F64, B.PL_MLP_F64
    assert B.pl_lattice_bytes(p) > n32


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("tau", 0.5), ("tau", float("nan")),
                                         ("rho0", 0.0), ("storage", 7), ("mlp", 9), ("G", float("inf"))])
def test_invalid_params_rejected(lib, field, value):
    p = B.pl_params_default(16, 16)
    setattr(p, field, value)
    n = ctypes.c_size_t()
    assert lib.pl_lattice_bytes(ctypes.byref(p), ctypes.byref(n)) == B.PL_ERR_INVALID_ARG


def test_f64_storage_needs_f64_network(lib):
    p = B.pl_params_default(16, 16, storage=B.PL_F64)   # mlp stays BF16
    n = ctypes.c_size_t()
    assert lib.pl_lattice_bytes(ctypes.byref(p), ctypes.byref(n)) == B.PL_ERR_INVALID_ARG


def test_create_rejects_bad_buffers_without_touching_the_device(lib):
    p = B.pl_params_default(16, 16)
    need = B.pl_lattice_bytes(p)
    h = ctypes.c_void_p()
    # NULL buffer, misaligned buffer, too small buffer
    assert lib.pl_lattice_create(ctypes.byref(p), None, need, None, ctypes.byref(h)) == B.PL_ERR_INVALID_ARG
    assert lib.pl_lattice_create(ctypes.byref(p), ctypes.c_void_p(0x1000 + 8), need, None,
                                 ctypes.byref(h)) == B.PL_ERR_INVALID_ARG
    assert lib.pl_lattice_create(ctypes.byref(p), ctypes.c_void_p(0x1000), need - 1, None,
                                 ctypes.byref(h)) == B.PL_ERR_BUDGET


def test_null_handle_rejected(lib):
    for name in ("pl_step", "pl_apply_correction", "pl_lattice_status", "pl_destroy"):
        fn = getattr(lib, name)
        args = [None] + ([1] if name == "pl_step" else [])
        assert fn(*args) == B.PL_ERR_INVALID_ARG


def test_train_params_default_and_argument_checks(lib):
    tp = B.pl_train_params_default()
    assert (tp.lr, tp.beta1, tp.beta2, tp.eps) == (3e-4, 0.9, 0.999, 1e-8)     # Sec. III-B learning rate
    assert (tp.lambda_phys, tp.lambda_int, tp.alpha1, tp.alpha2) == (1.0, 1.0, 1.0, 1.0)
    assert tp.mode == B.PL_TRAIN_SIMT
    h = ctypes.c_void_p()
    # no lattice: refused before any device work
    assert lib.pl_trainer_create(None, ctypes.byref(tp), 10, ctypes.c_void_p(256), 1 << 20,
                                 ctypes.byref(h)) == B.PL_ERR_INVALID_ARG
    out = ctypes.c_size_t(0)
    p = B.pl_params_default(16, 16, mlp_in=11)
    assert lib.pl_trainer_bytes(ctypes.byref(p), 10, ctypes.byref(out)) == B.PL_ERR_INVALID_ARG   # 2-input network only
    p = B.pl_params_default(16, 16)
    assert lib.pl_trainer_bytes(ctypes.byref(p), 0, ctypes.byref(out)) == B.PL_ERR_INVALID_ARG
    assert lib.pl_train(None, 1) == B.PL_ERR_INVALID_ARG
    assert lib.pl_trainer_destroy(None) == B.PL_ERR_INVALID_ARG


def test_batch_sizes_follow_storage_and_job_count(lib):
    # arena bytes of one job: two population buffers and the per-cell scratch fields (density,
    # momentum, gradient, network output), without the single-lattice handle's own weights and
    # table, ordered by storage width like a single lattice's
    p = B.pl_params_default(128, 96)
    n32 = B.pl_batch_job_bytes(p)
    assert 2 * 9 * 128 * 96 * 4 + 7 * 128 * 96 * 4 <= n32 < B.pl_lattice_bytes(p)
    p.storage = B.PL_F16_OFFSET
    n16 = B.pl_batch_job_bytes(p)
    assert 2 * 10 * 128 * 96 * 2 <= n16 < n32
    p.storage, p.mlp = B.PL_F64, B.PL_MLP_F64
    assert B.pl_batch_job_bytes(p) > n32 >= 2 * 9 * 128 * 96 * 4
    # the head grows with the job table and not with anything else
    heads = [B.pl_batch_overhead_bytes(m) for m in (1, 2, 64, 256, 4096)]
    assert all(a < b for a, b in zip(heads, heads[1:]))
    out = ctypes.c_size_t(0)
    for m in (0, -1, (1 << 20) + 1):
        assert lib.pl_batch_overhead_bytes(m, ctypes.byref(out)) == B.PL_ERR_INVALID_ARG
    bad = B.pl_params_default(16, 16)
    bad.tau = 0.5
    assert lib.pl_batch_job_bytes(ctypes.byref(bad), ctypes.byref(out)) == B.PL_ERR_INVALID_ARG


@pytest.mark.parametrize("storage,mlp,K,max_jobs,addr,status", [
    (7, B.PL_MLP_BF16, 100, 8, 0x1000, B.PL_ERR_INVALID_ARG),                  # unknown storage
    (B.PL_F64, B.PL_MLP_BF16, 100, 8, 0x1000, B.PL_ERR_INVALID_ARG),           # FP64 storage needs the FP64 network
    (B.PL_F32, B.PL_MLP_F64, 100, 8, 0x1000, B.PL_ERR_INVALID_ARG),            # FP64 network only with FP64 storage
    (B.PL_F16_OFFSET, B.PL_MLP_BF16, 0, 8, 0x1000, B.PL_ERR_INVALID_ARG),      # K < 1
    (B.PL_F16_OFFSET, B.PL_MLP_BF16, 100, 0, 0x1000, B.PL_ERR_INVALID_ARG),    # no job slots
    (B.PL_F16_OFFSET, B.PL_MLP_BF16, 100, 8, 0x1000 + 8, B.PL_ERR_INVALID_ARG),  # misaligned buffer
    (B.PL_F16_OFFSET, B.PL_MLP_BF16, 100, 8, 0, B.PL_ERR_INVALID_ARG),         # NULL buffer
])
def test_batch_create_rejects_bad_arguments_without_touching_the_device(lib, storage, mlp, K, max_jobs, addr,
                                                                        status):
    h = ctypes.c_void_p()
    head = B.pl_batch_overhead_bytes(8)
    assert lib.pl_batch_create(storage, mlp, K, max_jobs, ctypes.c_void_p(addr), head + (1 << 20), None,
                               ctypes.byref(h)) == status
    assert h.value is None


def test_batch_create_refuses_a_buffer_below_its_head(lib):
    h = ctypes.c_void_p()
    head = B.pl_batch_overhead_bytes(8)
    assert lib.pl_batch_create(B.PL_F16_OFFSET, B.PL_MLP_BF16, 100, 8, ctypes.c_void_p(0x1000), head - 1, None,
                               ctypes.byref(h)) == B.PL_ERR_BUDGET
    assert h.value is None
    for name in ("pl_batch_advance", "pl_batch_destroy"):
        fn = getattr(lib, name)
        assert fn(*([None] + ([1] if name == "pl_batch_advance" else []))) == B.PL_ERR_INVALID_ARG


def _c_layout():
    """sizeof / offsetof of every ABI struct and the value of every #define constant, as the C
    compiler sees include/pinnlbm.h."""
    import shutil
    import subprocess
    import tempfile
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"pl_params": B.pl_params, "pl_droplet": B.pl_droplet, "pl_metric_record": B.pl_metric_record,
               "pl_job_result": B.pl_job_result, "pl_train_params": B.pl_train_params}
    consts = sorted(n for n in dir(B) if re.fullmatch(r"PL_[A-Z0-9_]+", n))
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pinnlbm.h"', "int main(void) {"]
    for s, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    for c in consts:
        lines.append('printf("%s %%ld\\n", (long)(%s));' % (c, c))
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    vals = {}
    for ln in out.splitlines():
        parts = ln.split()
        vals[" ".join(parts[:-1])] = int(parts[-1])
    return structs, consts, vals


def test_binding_structs_and_constants_match_the_header():
    structs, consts, c = _c_layout()
    for s, cls in structs.items():
        assert c["%s size" % s] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert c["%s.%s" % (s, f)] == getattr(cls, f).offset, (s, f)
    for name in consts:
        assert c[name] == getattr(B, name), name
    # the Python-side codes of the input generators are the header's
    assert (wl.F64, wl.F32, wl.F16_OFFSET) == (c["PL_F64"], c["PL_F32"], c["PL_F16_OFFSET"])
    assert (wl.MLP_F64, wl.MLP_F32, wl.MLP_BF16) == (c["PL_MLP_F64"], c["PL_MLP_F32"], c["PL_MLP_BF16"])

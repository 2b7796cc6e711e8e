"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, and exports
every entry point declared in include/fcgno.h; the oracle and the library stay separate."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    text = (ROOT / "include" / "fcgno.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fcgno_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_05598_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(str(libpath))
    syms = declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2402_05598_gb300 import fcgno
    assert sorted(fcgno.EXPORTS) == declared_symbols()


def test_host_only_calls(libpath):
    """Calls that need no GPU: status strings, weight counts, argument validation."""
    from paper_2402_05598_gb300 import fcgno
    from paper_2402_05598_gb300 import inputs as I
    assert fcgno.status_str(fcgno.FCGNO_OK) == "ok"
    assert "breakdown" in fcgno.status_str(fcgno.FCGNO_EBREAKDOWN)
    for C, M in ((16, 8), (32, 12)):
        d = fcgno.make_desc(width=C, layers=4, modes=M)
        assert fcgno.weight_count(d) == I.weight_count(I.ModelDesc(width=C, layers=4, modes=M, proj_width=C))
    bad = fcgno.make_desc(width=0)
    assert fcgno.weight_count(bad) == 0
    # invalid arguments are rejected before any CUDA call
    h = ctypes.c_void_p()
    assert fcgno.lib.fcgno_assemble(1, 1, None, None, ctypes.byref(h)) == fcgno.FCGNO_EINVAL
    opts = fcgno.fcgno_solve_opts(1e-6, 9, 10, 0, 1)
    assert fcgno.lib.fcgno_solve(None, None, None, None, ctypes.byref(opts), 1, None, None) == fcgno.FCGNO_EINVAL
    assert fcgno.workspace_bytes(64, 256, 1, fcgno.make_desc(32, 4, 12)) > 256 * 64 * 64 * 8 * 8


def test_oracle_and_library_do_not_import_each_other():
    for f in (ROOT / "oracle").rglob("*.py"):
        src = f.read_text()
        assert "paper_2402_05598_gb300" not in src, f
    for f in (ROOT / "paper_2402_05598_gb300").rglob("*.py"):
        src = f.read_text()
        assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
    for f in (ROOT / "paper_2402_05598_gb300" / "csrc").glob("*"):
        assert "oracle" not in f.read_text().lower(), f


def test_every_entry_rejects_bad_arguments_before_cuda(libpath):
    """Each C entry point checks its arguments before its first CUDA call: null handles and
    buffers, out-of-range sizes and modes give FCGNO_EINVAL and a last-error text naming the
    call, with no GPU present. Destroying a null handle is a no-op."""
    import numpy as np
    from paper_2402_05598_gb300 import fcgno as F
    L, EINVAL = F.lib, F.FCGNO_EINVAL
    h = ctypes.c_void_p()
    host = np.zeros(16)
    hp = host.ctypes.data
    opts = F.fcgno_solve_opts(1e-6, 1, 10, 0, 1)
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    w32 = np.zeros(8, dtype=np.float32)

    def rejects(rc, name):
        assert rc == EINVAL, (name, rc)
        assert name in F.last_error(), (name, F.last_error())

    for N, B, k, out in ((1, 1, hp, h), (4, 0, hp, h), (4, 1, None, h), (4, 1, hp, None)):
        rejects(L.fcgno_assemble(N, B, k, None, ctypes.byref(out) if out is not None else None), "fcgno_assemble")
    rejects(L.fcgno_apply_A(None, hp, hp, None), "fcgno_apply_A")
    rejects(L.fcgno_reassemble(None, hp, None), "fcgno_reassemble")
    rejects(L.fcgno_residual_pair(None, hp, hp, hp, hp, hp, None), "fcgno_residual_pair")
    rejects(L.fcgno_reassemble(ctypes.c_void_p(1), None, None), "fcgno_reassemble")
    rejects(L.fcgno_model_create(ctypes.byref(F.make_desc(width=0)), w32.ctypes.data, None, ctypes.byref(h)),
            "fcgno_model_create")
    rejects(L.fcgno_model_create(ctypes.byref(F.make_desc()), None, None, ctypes.byref(h)), "fcgno_model_create")
    rejects(L.fcgno_model_sync(None, None), "fcgno_model_sync")
    for mode in (0, 3, -1):
        rejects(L.fcgno_model_set_train_recompute(None, mode), "fcgno_model_set_train_recompute")
    rejects(L.fcgno_precond_apply(None, None, hp, hp, F.PREC["bf16"], None), "fcgno_precond_apply")
    rejects(L.fcgno_solve(None, None, hp, hp, ctypes.byref(opts), F.PREC["fp64"], None, None), "fcgno_solve")
    for steps in (0, 65):
        rejects(L.fcgno_solve_jacobi(None, steps, hp, hp, ctypes.byref(opts), None, None), "fcgno_solve_jacobi")
    rejects(L.fcgno_solve_host(1, 1, hp, hp, hp, None, ctypes.byref(opts), F.PREC["fp64"], None, None),
            "fcgno_solve_host")
    rejects(L.fcgno_solve_host(4, 0, hp, hp, hp, None, ctypes.byref(opts), F.PREC["fp64"], None, None),
            "fcgno_solve_host")
    # options and precision are checked before the host buffers are copied anywhere
    bad_opts = [F.fcgno_solve_opts(-1.0, 1, 10, 0, 1), F.fcgno_solve_opts(1e-6, 0, 10, 0, 1),
                F.fcgno_solve_opts(1e-6, 9, 10, 0, 1), F.fcgno_solve_opts(1e-6, 1, -1, 0, 1)]
    for o in bad_opts:
        rejects(L.fcgno_solve_host(4, 1, hp, hp, hp, None, ctypes.byref(o), F.PREC["fp64"], None, None), "fcgno_solve")
    rejects(L.fcgno_solve_host(4, 1, hp, hp, hp, None, None, F.PREC["fp64"], None, None), "fcgno_solve")
    rejects(L.fcgno_solve_host(4, 1, hp, hp, hp, None, ctypes.byref(opts), 7, None, None), "fcgno_solve_host")
    rejects(L.fcgno_krylov_harvest(None, hp, hp, hp, 0, hp, hp, None, None), "fcgno_krylov_harvest")
    rejects(L.fcgno_train_step_loss(None, None, hp, hp, 1, F.PREC["fp64"], 0, hp, hp, None), "fcgno_train_step")
    rejects(L.fcgno_train_step_f64(None, None, hp, hp, 1, 0, hp, hp, None), "fcgno_train_step_f64")
    for blocks, steps in ((0, 1), (1, 0), ((1 << 20) + 1, 1), (1, (1 << 24) + 1)):
        rejects(L.fcgno_fp64_fma_rate(blocks, steps, 1.0, 0.0, hp, ctypes.byref(n), None), "fcgno_fp64_fma_rate")
    rejects(L.fcgno_fp64_fma_rate(1, 1, 1.0, 0.0, hp, None, None), "fcgno_fp64_fma_rate")
    bucket_bad = [(1, 4, 1, 1e-6, 10, 8), (64, 0, 1, 1e-6, 10, 8), (64, 4, 0, 1e-6, 10, 8), (64, 4, 9, 1e-6, 10, 8),
                  (64, 4, 1, -1.0, 10, 8), (64, 4, 1, float("nan"), 10, 8), (64, 4, 1, 1e-6, 0, 8),
                  (64, 4, 1, 1e-6, 10, 0)]
    for N, cap, m, tol, mi, g in bucket_bad:
        rejects(L.fcgno_bucket_create(N, cap, None, F.PREC["fp64"], m, tol, mi, g, None, ctypes.byref(h)),
                "fcgno_bucket_create")
    for prec in (-1, 4):
        rejects(L.fcgno_bucket_create(64, 4, None, prec, 1, 1e-6, 10, 8, None, ctypes.byref(h)), "fcgno_bucket_create")
    rejects(L.fcgno_bucket_admit(None, 0, hp, hp, hp, None), "fcgno_bucket_admit")
    rejects(L.fcgno_bucket_step(None, None), "fcgno_bucket_step")
    rejects(L.fcgno_bucket_poll(None, hp, hp, hp, None), "fcgno_bucket_poll")
    rejects(L.fcgno_bucket_take(None, 0, None, None), "fcgno_bucket_take")
    rejects(L.fcgno_bucket_serve_enable(None, 16, 16), "fcgno_bucket_serve_enable")
    rejects(L.fcgno_bucket_enqueue(None, None), "fcgno_bucket_enqueue")
    assert L.fcgno_bucket_results(None, None, 4) == -1
    rejects(L.fcgno_wait_selftest(None, 1e-3, None), "fcgno_wait_selftest")
    rejects(L.fcgno_set_launch_shape(3), "fcgno_set_launch_shape")
    rejects(L.fcgno_set_launch_shape(-1), "fcgno_set_launch_shape")
    rejects(L.fcgno_wait_selftest(ctypes.c_void_p(1), 0.0, None), "fcgno_wait_selftest")
    rejects(L.fcgno_wait_selftest(ctypes.c_void_p(1), 2.0, None), "fcgno_wait_selftest")
    rejects(L.fcgno_trace_collect(None, ctypes.byref(n)), "fcgno_trace_collect")
    rejects(L.fcgno_trace_collect(ctypes.byref(ms), None), "fcgno_trace_collect")
    for destroy in (L.fcgno_op_destroy, L.fcgno_model_destroy, L.fcgno_bucket_destroy):
        assert destroy(None) == F.FCGNO_OK


def test_precision_supported_query(libpath):
    """fcgno_precision_supported (host-only) states the shape rule the calls enforce: the
    CUDA-core precisions take any valid desc with N >= 2*modes, the 16-bit ones also need
    width 16 or 32, proj_width = width and N in {32, 64} or a multiple of 128."""
    from paper_2402_05598_gb300 import fcgno as F
    d32 = F.make_desc(32, 4, 12)
    d16 = F.make_desc(16, 4, 8)
    for N in (24, 33, 48, 64, 100, 128, 130, 256, 1024):
        for prec in ("fp64", "fp32"):
            assert F.precision_supported(N, d32, prec)
    for N, ok in ((32, True), (64, True), (128, True), (256, True), (2048, True),
                  (48, False), (96, False), (100, False), (130, False), (192, False)):
        for prec in ("bf16", "fp16"):
            assert F.precision_supported(N, d32, prec) == ok, (N, prec)
    assert F.precision_supported(32, d16, "bf16")
    assert not F.precision_supported(64, F.make_desc(24, 4, 12), "bf16")       # width 24
    assert not F.precision_supported(64, F.make_desc(32, 4, 12, 16), "bf16")   # proj_width != width
    assert F.precision_supported(64, F.make_desc(32, 4, 12, 16), "fp64")
    assert not F.precision_supported(22, d32, "fp64")                          # N < 2 * modes
    assert not F.precision_supported(64, F.make_desc(width=0), "fp64")
    assert F.lib.fcgno_precision_supported(64, ctypes.byref(d32), 9) == 0      # unknown precision
    assert F.lib.fcgno_precision_supported(64, None, 0) == 0

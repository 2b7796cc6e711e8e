"""Python binding of the C ABI in ``include/fcgno.h`` (ctypes; argument marshalling only).

Functions keep the C names. Tensors are passed as raw device pointers (torch tensors
must be contiguous float64/float32 CUDA tensors). Every computation happens inside
``libfcgno.so``; importing this module on a machine without the built library raises.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_size_t, c_uint64, c_void_p
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libfcgno.so"

FCGNO_OK, FCGNO_EINVAL, FCGNO_ENOMEM, FCGNO_ECUDA, FCGNO_ENOCONV, FCGNO_EBREAKDOWN, FCGNO_ETIMEOUT = range(7)
FCGNO_FP64, FCGNO_BF16, FCGNO_FP16, FCGNO_FP32 = range(4)
PREC = {"fp64": FCGNO_FP64, "bf16": FCGNO_BF16, "fp16": FCGNO_FP16, "fp32": FCGNO_FP32}
FCGNO_LOSS_ENERGY, FCGNO_LOSS_L2 = range(2)
LOSS = {"energy": FCGNO_LOSS_ENERGY, "l2": FCGNO_LOSS_L2}


class fcgno_model_desc(Structure):
    """fcgno_model_desc of the C ABI: width C, layers L, modes M, proj_width C_p, in_channels (2),
    output_scale (0: h^2 rms(r); 1: h^2 rms(r) / k)."""
    _fields_ = [("width", c_int), ("layers", c_int), ("modes", c_int), ("proj_width", c_int), ("in_channels", c_int),
                ("output_scale", c_int)]


class fcgno_solve_opts(Structure):
    """fcgno_solve_opts of the C ABI: tol, m_max, max_iter, fixed_iters, check_every."""
    _fields_ = [("tol", c_double), ("m_max", c_int), ("max_iter", c_int), ("fixed_iters", c_int),
                ("check_every", c_int)]


class fcgno_solve_info(Structure):
    """fcgno_solve_info of the C ABI: per-instance iterations, status, relative residual, ||r_0||."""
    _fields_ = [("iters", c_int32), ("status", c_int32), ("relres", c_double), ("r0norm", c_double)]


class fcgno_serve_request(Structure):
    """fcgno_serve_request of the C ABI: device pointers k, f, x0, x_out ([N][N] float64) and a tag."""
    _fields_ = [("k", c_void_p), ("f", c_void_p), ("x0", c_void_p), ("x_out", c_void_p), ("tag", c_uint64)]


class fcgno_serve_result(Structure):
    """fcgno_serve_result of the C ABI: tag, status, iterations, relative residual, publication number."""
    _fields_ = [("tag", c_uint64), ("status", c_int32), ("iters", c_int32), ("relres", c_double), ("seq", c_uint64)]


class FcgnoError(RuntimeError):
    """A non-OK fcgno_status; `code` holds it, the message the call and fcgno_last_error()."""
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_str(code)} ({last_error()})")
        self.code = code


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build() (the library has no CPU fallback)")
    lib = ctypes.CDLL(str(_LIB_PATH))
    P = c_void_p
    sig = {
        "fcgno_assemble": (c_int, [c_int, c_int, P, P, POINTER(P)]),
        "fcgno_reassemble": (c_int, [P, P, P]),
        "fcgno_op_destroy": (c_int, [P]),
        "fcgno_apply_A": (c_int, [P, P, P, P]),
        "fcgno_residual_pair": (c_int, [P, P, P, P, P, P, P]),
        "fcgno_weight_count": (c_size_t, [POINTER(fcgno_model_desc)]),
        "fcgno_model_create": (c_int, [POINTER(fcgno_model_desc), P, P, POINTER(P)]),
        "fcgno_model_sync": (c_int, [P, P]),
        "fcgno_model_destroy": (c_int, [P]),
        "fcgno_precond_apply": (c_int, [P, P, P, P, c_int, P]),
        "fcgno_solve": (c_int, [P, P, P, P, POINTER(fcgno_solve_opts), c_int, POINTER(fcgno_solve_info), P]),
        "fcgno_solve_host": (c_int, [c_int, c_int, P, P, P, P, POINTER(fcgno_solve_opts), c_int,
                                     POINTER(fcgno_solve_info), P]),
        "fcgno_solve_host_release": (c_int, []),
        "fcgno_solve_noalloc": (c_int, [P, P, P, POINTER(fcgno_solve_opts), POINTER(fcgno_solve_info), P]),
        "fcgno_solve_jacobi": (c_int, [P, c_int, P, P, POINTER(fcgno_solve_opts), POINTER(fcgno_solve_info), P]),
        "fcgno_krylov_harvest": (c_int, [P, P, P, P, c_int, P, P, POINTER(fcgno_solve_info), P]),
        "fcgno_train_step": (c_int, [P, P, P, P, c_int, c_int, P, P, P]),
        "fcgno_train_step_loss": (c_int, [P, P, P, P, c_int, c_int, c_int, P, P, P]),
        "fcgno_train_step_f64": (c_int, [P, P, P, P, c_int, c_int, P, P, P]),
        "fcgno_model_set_train_recompute": (c_int, [P, c_int]),
        "fcgno_workspace_bytes": (c_size_t, [c_int, c_int, c_int, POINTER(fcgno_model_desc), c_int]),
        "fcgno_precision_supported": (c_int, [c_int, POINTER(fcgno_model_desc), c_int]),
        "fcgno_status_str": (c_char_p, [c_int]),
        "fcgno_last_error": (c_char_p, []),
        "fcgno_launch_count": (c_uint64, []),
        "fcgno_fp64_fma_rate": (c_int, [c_int, c_int, c_double, c_double, P, POINTER(c_uint64), P]),
        "fcgno_bucket_create": (c_int, [c_int, c_int, P, c_int, c_int, c_double, c_int, c_int, P, POINTER(P)]),
        "fcgno_bucket_admit": (c_int, [P, c_int, P, P, P, P]),
        "fcgno_bucket_step": (c_int, [P, P]),
        "fcgno_bucket_poll": (c_int, [P, P, P, P, P]),
        "fcgno_bucket_take": (c_int, [P, c_int, P, P]),
        "fcgno_bucket_destroy": (c_int, [P]),
        "fcgno_bucket_serve_enable": (c_int, [P, c_int, c_int]),
        "fcgno_bucket_enqueue": (c_int, [P, POINTER(fcgno_serve_request)]),
        "fcgno_bucket_results": (c_int, [P, POINTER(fcgno_serve_result), c_int]),
        "fcgno_wait_selftest": (c_int, [P, c_double, P]),
        "fcgno_set_launch_shape": (c_int, [c_int]),
        "fcgno_trace_set": (c_int, [c_char_p]),
        "fcgno_trace_collect": (c_int, [POINTER(c_double), POINTER(c_uint64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# Exported symbol names, in the order of include/fcgno.h.
EXPORTS = [
    "fcgno_assemble", "fcgno_reassemble", "fcgno_op_destroy", "fcgno_apply_A", "fcgno_residual_pair", "fcgno_weight_count", "fcgno_model_create",
    "fcgno_model_sync", "fcgno_model_destroy", "fcgno_precond_apply", "fcgno_solve", "fcgno_solve_host",
    "fcgno_solve_host_release",
    "fcgno_solve_noalloc", "fcgno_solve_jacobi", "fcgno_krylov_harvest", "fcgno_train_step", "fcgno_train_step_loss",
    "fcgno_model_set_train_recompute", "fcgno_train_step_f64", "fcgno_workspace_bytes", "fcgno_precision_supported", "fcgno_status_str",
    "fcgno_last_error", "fcgno_launch_count", "fcgno_fp64_fma_rate", "fcgno_wait_selftest", "fcgno_set_launch_shape", "fcgno_trace_set",
    "fcgno_trace_collect",
    "fcgno_bucket_create", "fcgno_bucket_admit", "fcgno_bucket_step", "fcgno_bucket_poll", "fcgno_bucket_take",
    "fcgno_bucket_destroy", "fcgno_bucket_serve_enable", "fcgno_bucket_enqueue", "fcgno_bucket_results",
]


def precision_supported(N: int, desc: fcgno_model_desc, prec: str) -> bool:
    """Whether the preconditioner in `prec` supports this model shape on an N x N grid."""
    return bool(lib.fcgno_precision_supported(int(N), ctypes.byref(desc), PREC[prec]))


def status_str(code: int) -> str:
    """fcgno_status_str: static text of a status."""
    return lib.fcgno_status_str(code).decode()


def last_error() -> str:
    """fcgno_last_error: the calling thread's last error text."""
    return lib.fcgno_last_error().decode()


def launch_count() -> int:
    """fcgno_launch_count: this library's kernel launches since load."""
    return int(lib.fcgno_launch_count())


def fp64_fma_rate(blocks: int, steps: int, a: float, c: float, out, stream=None) -> int:
    """Launch the FP64 multiply-add rate kernel (out: blocks * 256 float64 on the device);
    returns the number of multiply-adds the launch performs. Time it with CUDA events."""
    n = c_uint64()
    _check(lib.fcgno_fp64_fma_rate(int(blocks), int(steps), float(a), float(c), _ptr(out), ctypes.byref(n),
                                   _stream(stream)), "fcgno_fp64_fma_rate")
    return int(n.value)


def wait_selftest(op: "Operator", limit_seconds: float, stream=None) -> int:
    """fcgno_wait_selftest: a bounded wait on a barrier nothing completes; returns the status
    code (FCGNO_ETIMEOUT when the wait gave up) instead of raising for it."""
    code = lib.fcgno_wait_selftest(op.handle, float(limit_seconds), _stream(stream))
    if code not in (FCGNO_OK, FCGNO_ETIMEOUT):
        raise FcgnoError(code, "fcgno_wait_selftest")
    return code


def set_launch_shape(mode: str):
    """fcgno_set_launch_shape: "auto", "wide" or "narrow"."""
    _check(lib.fcgno_set_launch_shape({"auto": 0, "wide": 1, "narrow": 2}[mode]), "fcgno_set_launch_shape")


def trace_set(family: str):
    """Select the kernel family whose launches are bracketed by CUDA events ("" = off)."""
    _check(lib.fcgno_trace_set(family.encode()), "fcgno_trace_set")


def trace_collect():
    """(total device ms, traced launches) since the previous collect."""
    ms = c_double()
    cnt = c_uint64()
    _check(lib.fcgno_trace_collect(ctypes.byref(ms), ctypes.byref(cnt)), "fcgno_trace_collect")
    return float(ms.value), int(cnt.value)


def _check(code: int, where: str):
    if code != FCGNO_OK:
        raise FcgnoError(code, where)


def _ptr(t) -> int:
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def make_desc(width=32, layers=4, modes=12, proj_width=None, in_channels=2, output_scale=0) -> fcgno_model_desc:
    """A fcgno_model_desc (proj_width defaults to width)."""
    return fcgno_model_desc(width, layers, modes, proj_width if proj_width is not None else width, in_channels,
                            output_scale)


def weight_count(desc: fcgno_model_desc) -> int:
    """fcgno_weight_count: float32 elements of the weight blob (0 for an invalid desc)."""
    return int(lib.fcgno_weight_count(ctypes.byref(desc)))


class Operator:
    """fcgno_assemble handle over a [B][N][N] float64 CUDA tensor k."""

    def __init__(self, k, stream=None):
        import torch
        assert k.dtype == torch.float64 and k.is_cuda and k.dim() == 3 and k.shape[1] == k.shape[2]
        self.B, self.N = int(k.shape[0]), int(k.shape[1])
        self.handle = c_void_p()
        _check(lib.fcgno_assemble(self.N, self.B, _ptr(k), _stream(stream), ctypes.byref(self.handle)),
               "fcgno_assemble")

    def reassemble(self, k, stream=None):
        """fcgno_reassemble: new coefficient fields (same N and batch) into this operator."""
        assert k.dtype == __import__("torch").float64 and tuple(k.shape) == (self.B, self.N, self.N)
        _check(lib.fcgno_reassemble(self.handle, _ptr(k), _stream(stream)), "fcgno_reassemble")

    def apply(self, x, y, stream=None):
        """fcgno_apply_A: y = A x for every instance."""
        _check(lib.fcgno_apply_A(self.handle, _ptr(x), _ptr(y), _stream(stream)), "fcgno_apply_A")

    def residual_pair(self, b, u, u_star, r_out, e_out, stream=None):
        """fcgno_residual_pair: r_out = b - A u, e_out = u_star - u for every instance."""
        _check(lib.fcgno_residual_pair(self.handle, _ptr(b), _ptr(u), _ptr(u_star), _ptr(r_out), _ptr(e_out),
                                       _stream(stream)), "fcgno_residual_pair")

    def close(self):
        if self.handle:
            lib.fcgno_op_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """fcgno_model_create handle; keeps a reference to the float32 CUDA weight blob."""

    def __init__(self, desc: fcgno_model_desc, weights, stream=None):
        import torch
        assert weights.dtype == torch.float32 and weights.is_cuda and weights.numel() == weight_count(desc)
        self.desc = desc
        self.weights = weights
        self.handle = c_void_p()
        _check(lib.fcgno_model_create(ctypes.byref(desc), _ptr(weights), _stream(stream), ctypes.byref(self.handle)),
               "fcgno_model_create")

    def sync(self, stream=None):
        _check(lib.fcgno_model_sync(self.handle, _stream(stream)), "fcgno_model_sync")

    def set_train_recompute(self, mode: str):
        """Activation checkpointing of training steps: "auto", "always" or "never"."""
        code = {"auto": 0, "always": 1, "never": 2}[mode]
        _check(lib.fcgno_model_set_train_recompute(self.handle, code), "fcgno_model_set_train_recompute")

    def close(self):
        if self.handle:
            lib.fcgno_model_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def precond_apply(model: Model, op: Operator, r, z, prec="bf16", stream=None):
    """fcgno_precond_apply: z = NO(r, log k) for every instance of op, in precision `prec`."""
    _check(lib.fcgno_precond_apply(model.handle, op.handle, _ptr(r), _ptr(z), PREC[prec], _stream(stream)),
           "fcgno_precond_apply")


def _opts(tol, m_max, max_iter, fixed_iters, check_every):
    return fcgno_solve_opts(float(tol), int(m_max), int(max_iter), int(bool(fixed_iters)), int(check_every))


def _info_list(arr):
    return [{"iters": int(i.iters), "status": int(i.status), "relres": float(i.relres), "r0norm": float(i.r0norm)}
            for i in arr]


def solve(op: Operator, model, b, x, tol=1e-6, m_max=1, max_iter=1000, prec="bf16", fixed_iters=False,
          check_every=8, stream=None):
    """fcgno_solve: x (u_0 on entry) is overwritten with the iterate; returns per-instance info."""
    info = (fcgno_solve_info * op.B)()
    opts = _opts(tol, m_max, max_iter, fixed_iters, check_every)
    _check(lib.fcgno_solve(op.handle, model.handle if model is not None else None, _ptr(b), _ptr(x),
                           ctypes.byref(opts), PREC[prec], info, _stream(stream)), "fcgno_solve")
    return _info_list(info)


def solve_host(k: np.ndarray, b: np.ndarray, x: np.ndarray, model=None, tol=1e-6, m_max=1, max_iter=1000,
               prec="bf16", fixed_iters=False, check_every=8, stream=None):
    """fcgno_solve_host on host float64 arrays [B][N][N] (x overwritten in place)."""
    for a in (k, b, x):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == k.shape
    B, N = k.shape[0], k.shape[1]
    info = (fcgno_solve_info * B)()
    opts = _opts(tol, m_max, max_iter, fixed_iters, check_every)
    _check(lib.fcgno_solve_host(N, B, k.ctypes.data, b.ctypes.data, x.ctypes.data,
                                model.handle if model is not None else None, ctypes.byref(opts), PREC[prec], info,
                                _stream(stream)), "fcgno_solve_host")
    return _info_list(info)


def solve_host_release():
    """fcgno_solve_host_release: frees the device state fcgno_solve_host keeps between calls."""
    _check(lib.fcgno_solve_host_release(), "fcgno_solve_host_release")


def solve_jacobi(op: Operator, steps, b, x, tol=1e-6, m_max=1, max_iter=1000, fixed_iters=False, check_every=8,
                 stream=None):
    """fcgno_solve_jacobi: Algorithm 1 with the Jacobi(steps) preconditioner (Eq. (15))."""
    info = (fcgno_solve_info * op.B)()
    opts = _opts(tol, m_max, max_iter, fixed_iters, check_every)
    _check(lib.fcgno_solve_jacobi(op.handle, int(steps), _ptr(b), _ptr(x), ctypes.byref(opts), info,
                                  _stream(stream)), "fcgno_solve_jacobi")
    return _info_list(info)


def solve_noalloc(op: Operator, b, x, tol=1e-6, m_max=1, max_iter=1000, fixed_iters=False, check_every=8,
                  stream=None):
    """fcgno_solve_noalloc: identity-preconditioned solve with no device allocation (for callers
    that cannot allocate); its state lives in the library's fixed 8 MiB device array."""
    info = (fcgno_solve_info * op.B)()
    opts = _opts(tol, m_max, max_iter, fixed_iters, check_every)
    _check(lib.fcgno_solve_noalloc(op.handle, _ptr(b), _ptr(x), ctypes.byref(opts), info, _stream(stream)),
           "fcgno_solve_noalloc")
    return _info_list(info)


def krylov_harvest(op: Operator, b, x0, u_star, K, r_out, e_out, stream=None):
    """fcgno_krylov_harvest: K CG iterates per instance as (r_i, e_i = u_star - u_i) pairs."""
    info = (fcgno_solve_info * op.B)()
    _check(lib.fcgno_krylov_harvest(op.handle, _ptr(b), _ptr(x0), _ptr(u_star), int(K), _ptr(r_out), _ptr(e_out),
                                    info, _stream(stream)), "fcgno_krylov_harvest")
    return _info_list(info)


def train_step(model: Model, op: Operator, r, e, loss, grad, prec="fp32", stream=None, loss_kind="energy"):
    """One step of Eq. (11) (loss_kind "energy") or of the L2 ablation loss ("l2")."""
    if loss_kind == "energy":
        _check(lib.fcgno_train_step(model.handle, op.handle, _ptr(r), _ptr(e), op.B, PREC[prec], _ptr(loss),
                                    _ptr(grad), _stream(stream)), "fcgno_train_step")
    else:
        _check(lib.fcgno_train_step_loss(model.handle, op.handle, _ptr(r), _ptr(e), op.B, PREC[prec],
                                         LOSS[loss_kind], _ptr(loss), _ptr(grad), _stream(stream)),
               "fcgno_train_step_loss")


def train_step_f64(model: Model, op: Operator, r, e, loss, grad, stream=None, loss_kind="energy"):
    """fcgno_train_step_f64: the FP64 step with loss and gradient stored in FP64 (float64 tensors)."""
    _check(lib.fcgno_train_step_f64(model.handle, op.handle, _ptr(r), _ptr(e), op.B, LOSS[loss_kind], _ptr(loss),
                                    _ptr(grad), _stream(stream)), "fcgno_train_step_f64")


def workspace_bytes(N, batch, m_max, desc, prec="bf16") -> int:
    """fcgno_workspace_bytes: device bytes a solve of this shape needs (for HBM admission)."""
    return int(lib.fcgno_workspace_bytes(int(N), int(batch), int(m_max), ctypes.byref(desc), PREC[prec]))


class Bucket:
    """fcgno_bucket_*: a resident batch of same-size solves with independent slots."""

    def __init__(self, N, capacity, model=None, prec="bf16", m_max=1, tol=1e-6, max_iter=1000, iters_per_step=8,
                 stream=None):
        self.N, self.capacity = int(N), int(capacity)
        self.handle = c_void_p()
        _check(lib.fcgno_bucket_create(self.N, self.capacity, model.handle if model is not None else None, PREC[prec],
                                       int(m_max), float(tol), int(max_iter), int(iters_per_step), _stream(stream),
                                       ctypes.byref(self.handle)), "fcgno_bucket_create")
        self._status = np.zeros(self.capacity, dtype=np.int32)
        self._iters = np.zeros(self.capacity, dtype=np.int32)
        self._relres = np.zeros(self.capacity, dtype=np.float64)

    def admit(self, slot, k, f, x0, stream=None):
        """fcgno_bucket_admit: start a solve (k, f, x0: device [N][N]) in a free slot."""
        _check(lib.fcgno_bucket_admit(self.handle, int(slot), _ptr(k), _ptr(f), _ptr(x0), _stream(stream)),
               "fcgno_bucket_admit")

    def step(self, stream=None):
        """fcgno_bucket_step: advance every running slot by iters_per_step iterations."""
        _check(lib.fcgno_bucket_step(self.handle, _stream(stream)), "fcgno_bucket_step")

    def poll(self, stream=None):
        """fcgno_bucket_poll: (status, iterations, relative residual) per slot; synchronises."""
        _check(lib.fcgno_bucket_poll(self.handle, self._status.ctypes.data, self._iters.ctypes.data,
                                     self._relres.ctypes.data, _stream(stream)), "fcgno_bucket_poll")
        return self._status.copy(), self._iters.copy(), self._relres.copy()

    def take(self, slot, x_out=None, stream=None):
        """fcgno_bucket_take: copy the slot's iterate to x_out (optional) and free the slot."""
        _check(lib.fcgno_bucket_take(self.handle, int(slot), _ptr(x_out) if x_out is not None else None,
                                     _stream(stream)), "fcgno_bucket_take")

    def serve_enable(self, queue_capacity=4096, result_capacity=4096):
        """fcgno_bucket_serve_enable: admission and retirement move onto the device (a mapped
        request queue and result ring); use enqueue/step/results from then on."""
        _check(lib.fcgno_bucket_serve_enable(self.handle, int(queue_capacity), int(result_capacity)),
               "fcgno_bucket_serve_enable")
        self._res = (fcgno_serve_result * int(result_capacity))()
        self._keep = {}

    def enqueue(self, k, f, x0, x_out, tag) -> bool:
        """fcgno_bucket_enqueue (host-only); False when the queue is full. The tensors are kept
        alive here until the request's result has been collected."""
        req = fcgno_serve_request(_ptr(k), _ptr(f), _ptr(x0), _ptr(x_out), int(tag))
        code = lib.fcgno_bucket_enqueue(self.handle, ctypes.byref(req))
        if code == FCGNO_ENOMEM:
            return False
        _check(code, "fcgno_bucket_enqueue")
        self._keep[int(tag)] = (k, f, x0, x_out)
        return True

    def results(self):
        """fcgno_bucket_results (host-only): [(tag, status, iters, relres)] published since the last call."""
        n = lib.fcgno_bucket_results(self.handle, self._res, len(self._res))
        if n < 0:
            raise FcgnoError(FCGNO_EINVAL, "fcgno_bucket_results")
        out = []
        for i in range(n):
            r = self._res[i]
            out.append((int(r.tag), int(r.status), int(r.iters), float(r.relres)))
            self._keep.pop(int(r.tag), None)
        return out

    def close(self):
        if self.handle:
            lib.fcgno_bucket_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

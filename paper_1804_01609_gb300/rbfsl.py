"""Thin Python binding of librbfsl (include/rbfsl.h): argument marshalling only.

Every function here has the name of the C entry point it calls. Tensors are torch tensors
on the CUDA device (PyTorch provides device memory and streams); all computation happens
in the library's kernels. There is no fallback: if the CUDA library is missing or fails to
load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOTCONF, ENOMEM, ESINGULAR, EUNCOVERED, ETIMEDOUT, ECUDA, EKNN = 0, -1, -2, -3, -4, -5, -6, -7, -8
VEL_RIGID, VEL_DEFORM_Y2, VEL_NL = 0, 1, 2
LOCAL, GLOBAL, PU = 0, 1, 2
DIRECT, CENTER = 0, 1
PHS, GAUSS, IMQ = 0, 1, 2
FP64, MIXED = 0, 1
RK4, RK5 = 4, 5
GLOBAL_SOLVE, GLOBAL_CARDINAL = 0, 1
GLOBAL_EVAL_PAIRS, GLOBAL_EVAL_TC = 0, 1
F64, F32, F32X2 = 0, 1, 2
HOST, DEVICE = 0, 1
PU_WENDLAND, PU_BSPLINE = 0, 1

_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOTCONF: "ENOTCONF", ENOMEM: "ENOMEM",
          ESINGULAR: "ESINGULAR", EUNCOVERED: "EUNCOVERED", ETIMEDOUT: "ETIMEDOUT",
          ECUDA: "ECUDA", EKNN: "EKNN"}


class RbfslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


class Stats(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int64), ("singular_points", ctypes.c_int64),
                ("knn_failures", ctypes.c_int64), ("uncovered_points", ctypes.c_int64),
                ("time", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("device_timeouts", ctypes.c_int64), ("global_cholesky", ctypes.c_int64)]


SIGNATURES = {
    "rbfsl_version": (ctypes.c_char_p, []),
    "rbfsl_fp64_fma_rate": (_I, [_I64, _P, _P]),
    "rbfsl_last_error": (ctypes.c_char_p, [_P]),
    "rbfsl_trace_rk4": (_I, [_P, _I64, _I, _P, _D, _D, _I, _P, _P]),
    "rbfsl_trace_rk5": (_I, [_P, _I64, _I, _P, _D, _D, _I, _P, _P]),
    "rbfsl_set_integrator": (_I, [_P, _I]),
    "rbfsl_knn_index_create": (_I, [_P, _P, _I64, _I, _P]),
    "rbfsl_knn_index_destroy": (_I, [_P]),
    "rbfsl_knn_query": (_I, [_P, _P, _I64, _I, _P, _P, _P]),
    "rbfsl_stencil_weights": (_I, [_P, _I64, _P, _I64, _I, _I, _I, _D, _P, _P, _I, _P, _P]),
    "rbfsl_gather_dot": (_I, [_P, _P, _I64, _I, _P, _I, _I, _P, _P]),
    "rbfsl_global_factor": (_I, [_P, _I64, _I, _D, _P, _P, _P]),
    "rbfsl_global_factor_noalloc": (_I, [_P, _I64, _I, _D, _P, _P, _P]),
    "rbfsl_global_factor_chol": (_I, [_P, _I64, _I, _D, _P, _P, _P]),
    "rbfsl_global_solve": (_I, [_P, _P, _I64, _P, _I, _P, _P]),
    "rbfsl_global_eval": (_I, [_P, _I64, _P, _I64, _I, _D, _P, _I, _I, _P, _P]),
    "rbfsl_global_eval_tc_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I]),
    "rbfsl_global_eval_tc": (_I, [_P, _I64, _P, _I64, _I, _D, _P, _I, _I, _P, _P, ctypes.c_size_t, _P, _P]),
    "rbfsl_global_cardinal": (_I, [_P, _P, _P, _I64, _I, _D, _P, _I64, _P, _I, _P]),
    "rbfsl_cardinal_apply_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I]),
    "rbfsl_cardinal_apply": (_I, [_P, _I64, _I64, _P, _I, _I, _P, _P, ctypes.c_size_t, _P]),
    "rbfsl_set_global_form": (_I, [_P, _I]),
    "rbfsl_set_global_eval": (_I, [_P, _I]),
    "rbfsl_global_eval_pairs_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I]),
    "rbfsl_global_eval_pairs": (_I, [_P, _I64, _P, _I64, _I, _D, _P, _I, _P, _P, ctypes.c_size_t, _P]),
    "rbfsl_pu_create": (_I, [_P, _P, _I64, _P, _I64, _D, _I, _I, _D, _P]),
    "rbfsl_pu_destroy": (_I, [_P]),
    "rbfsl_pu_apply": (_I, [_P, _P, _I, _P, _I64, _I, _I, _P, _P, _P]),
    "rbfsl_set_pu": (_I, [_P, _P, _I64, _D, _I, _I]),
    "rbfsl_batch_create": (_I, [_P, _I, _P]),
    "rbfsl_batch_destroy": (_I, [_P]),
    "rbfsl_batch_add": (_I, [_P, _P, _P]),
    "rbfsl_batch_remove": (_I, [_P, _I]),
    "rbfsl_batch_step": (_I, [_P, _I]),
    "rbfsl_batch_get_q": (_I, [_P, _I, _P]),
    "rbfsl_batch_problem_stats": (_I, [_P, _I, _P]),
    "rbfsl_batch_set_graph": (_I, [_P, _I]),
    "rbfsl_batch_autotune": (_I, [_P, _P, _I]),
    "rbfsl_server_create": (_I, [_P, _I, ctypes.c_size_t, _I]),
    "rbfsl_server_destroy": (_I, [_P]),
    "rbfsl_server_submit": (_I, [_P, _P, _P]),
    "rbfsl_server_poll": (_I, [_P, ctypes.c_uint64, _P]),
    "rbfsl_server_result": (_I, [_P, ctypes.c_uint64, _P, _P]),
    "rbfsl_server_wait_idle": (_I, [_P, _D]),
    "rbfsl_server_info": (_I, [_P, _P]),
    "rbfsl_create": (_I, [_P, _I, _P]),
    "rbfsl_destroy": (_I, [_P]),
    "rbfsl_set_nodes": (_I, [_P, _P, _I64, _I]),
    "rbfsl_set_velocity": (_I, [_P, _I, _P, _I]),
    "rbfsl_set_method": (_I, [_P, _I, _I]),
    "rbfsl_set_stencil_size": (_I, [_P, _I]),
    "rbfsl_set_sh_degree": (_I, [_P, _I]),
    "rbfsl_set_kernel": (_I, [_P, _I, _D]),
    "rbfsl_set_precision": (_I, [_P, _I]),
    "rbfsl_set_dt": (_I, [_P, _D]),
    "rbfsl_set_time": (_I, [_P, _D]),
    "rbfsl_set_tracers": (_I, [_P, _P, _I64, _I, _I, _I]),
    "rbfsl_step": (_I, [_P, _I]),
    "rbfsl_get_q": (_I, [_P, _P, _I, _I]),
    "rbfsl_get_stats": (_I, [_P, _P]),
    "rbfsl_last_step_buffers": (_I, [_P, _P, _P, _P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load librbfsl.so (building it first if asked); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != OK:
        msg = load().rbfsl_last_error(ctx)
        raise RbfslError(rc, msg.decode() if msg else "")
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


# --------------------------------------------------------------------------- stateless ops
def rbfsl_fp64_fma_rate(iters=1 << 16, stream=None):
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    v = ctypes.c_double(0.0)
    _check(load().rbfsl_fp64_fma_rate(iters, ctypes.byref(v), _stream(stream)))
    return v.value


def rbfsl_trace_rk4(x, vel_kind, vel_params, t1, dt, precision, xi, stream=None):
    prm = np.ascontiguousarray(vel_params, dtype=np.float64)
    _check(load().rbfsl_trace_rk4(_ptr(x), x.shape[0], vel_kind, prm.ctypes.data, t1, dt,
                                  precision, _ptr(xi), _stream(stream)))


def rbfsl_trace_rk5(x, vel_kind, vel_params, t1, dt, precision, xi, stream=None):
    prm = np.ascontiguousarray(vel_params, dtype=np.float64)
    _check(load().rbfsl_trace_rk5(_ptr(x), x.shape[0], vel_kind, prm.ctypes.data, t1, dt,
                                  precision, _ptr(xi), _stream(stream)))


class KnnIndex:
    def __init__(self, x, k_hint, stream=None):
        self._h = ctypes.c_void_p()
        self.N = x.shape[0]
        _check(load().rbfsl_knn_index_create(ctypes.byref(self._h), _ptr(x), x.shape[0],
                                             k_hint, _stream(stream)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().rbfsl_knn_index_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbfsl_knn_index_create(x, k_hint, stream=None) -> KnnIndex:
    return KnnIndex(x, k_hint, stream)


def rbfsl_knn_query(index, q, k, idx, status=None, stream=None):
    _check(load().rbfsl_knn_query(index.handle, _ptr(q), q.shape[0], k, _ptr(idx),
                                  _ptr(status), _stream(stream)))


def _weights_code(w):
    """float64 / float32 N x n, or N x n x 2 float32 (FP32 pairs, RBFSL_F32X2)."""
    import torch
    if w.dim() == 3 and w.shape[2] == 2 and w.dtype == torch.float32:
        return F32X2
    return _dtype_code(w)


def rbfsl_stencil_weights(x, idx, n, ell, kernel, kparam, p, w, status=None, stream=None):
    _check(load().rbfsl_stencil_weights(_ptr(x), x.shape[0], _ptr(idx), p.shape[0], n, ell,
                                        kernel, float(kparam), _ptr(p), _ptr(w), _weights_code(w),
                                        _ptr(status), _stream(stream)))


def rbfsl_gather_dot(idx, w, q, q_out, stream=None, pairs=False):
    """pairs=True: w, q and q_out are FP32 pairs (Nq x n x 2, N x T x 2, Nq x T x 2 float32)."""
    if pairs:
        if q.dim() != 3 or q.shape[2] != 2 or _weights_code(w) != F32X2:
            raise ValueError("pairs=True wants q of shape N x T x 2 and w of shape Nq x n x 2 (float32)")
        T, code = q.shape[1], F32X2
    else:
        T, code = (q.shape[1] if q.dim() == 2 else 1), _dtype_code(q)
    _check(load().rbfsl_gather_dot(_ptr(idx), _ptr(w), idx.shape[0], idx.shape[1], _ptr(q), T,
                                   code, _ptr(q_out), _stream(stream)))


def rbfsl_global_factor(x, kernel, eps, LU, perm, stream=None):
    _check(load().rbfsl_global_factor(_ptr(x), x.shape[0], kernel, float(eps), _ptr(LU), _ptr(perm),
                                      _stream(stream)))


def rbfsl_global_factor_noalloc(x, kernel, eps, LU, perm, stream=None):
    """rbfsl_global_factor without any device allocation (scratch in a library-owned array)."""
    _check(load().rbfsl_global_factor_noalloc(_ptr(x), x.shape[0], kernel, float(eps), _ptr(LU),
                                              _ptr(perm), _stream(stream)))


def rbfsl_global_factor_chol(x, kernel, eps, LU, perm, stream=None):
    """Cholesky factor of A_X in rbfsl_global_factor's form (raises ESINGULAR on breakdown)."""
    _check(load().rbfsl_global_factor_chol(_ptr(x), x.shape[0], kernel, float(eps), _ptr(LU), _ptr(perm),
                                           _stream(stream)))


def rbfsl_global_solve(LU, perm, q, c, stream=None):
    T = q.shape[1] if q.dim() == 2 else 1
    _check(load().rbfsl_global_solve(_ptr(LU), _ptr(perm), q.shape[0], _ptr(q), T, _ptr(c),
                                     _stream(stream)))


def rbfsl_global_eval(p, x, kernel, eps, c, out, stream=None):
    T = c.shape[1] if c.dim() == 2 else 1
    _check(load().rbfsl_global_eval(_ptr(p), p.shape[0], _ptr(x), x.shape[0], kernel, float(eps),
                                    _ptr(c), T, _dtype_code(c), _ptr(out), _stream(stream)))


class PUPatches:
    """RBF-PU patches with their LU factors (rbfsl_pu_create / rbfsl_pu_destroy)."""

    def __init__(self, x, centers, radius, ell, kernel, kparam, stream=None):
        self._h = ctypes.c_void_p()
        _check(load().rbfsl_pu_create(ctypes.byref(self._h), _ptr(x), x.shape[0], _ptr(centers),
                                      centers.shape[0], float(radius), ell, kernel, float(kparam),
                                      _stream(stream)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().rbfsl_pu_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbfsl_pu_create(x, centers, radius, ell, kernel, kparam, stream=None) -> PUPatches:
    return PUPatches(x, centers, radius, ell, kernel, kparam, stream)


def rbfsl_pu_apply(pu, q, p, weight_kind, out, status=None, stream=None, pairs=False):
    """pairs=True: out holds FP32 pairs (Nq x T x 2 float32), the RBFSL_F32X2 evaluation."""
    T = q.shape[1] if q.dim() == 2 else 1
    if pairs:
        if out.dtype.itemsize != 4 or out.dim() != 3 or out.shape[2] != 2:
            raise ValueError("pairs=True wants out of shape Nq x T x 2 (float32)")
        code = F32X2
    else:
        code = _dtype_code(out)
    _check(load().rbfsl_pu_apply(pu.handle, _ptr(q), T, _ptr(p), p.shape[0], weight_kind,
                                 code, _ptr(out), _ptr(status), _stream(stream)))


class Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nodes", ctypes.c_void_p), ("n", ctypes.c_int),
                ("ell", ctypes.c_int), ("phs_power", ctypes.c_double), ("mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("vel_kind", ctypes.c_int),
                ("vel_params", ctypes.c_double * 4), ("t0", ctypes.c_double),
                ("dt", ctypes.c_double), ("T", ctypes.c_int), ("q0", ctypes.c_void_p)]


class Batch:
    """Many local problems stepped together (rbfsl_batch_*)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        self._keep = {}
        _check(load().rbfsl_batch_create(ctypes.byref(self._h), device,
                                         _stream(stream) if stream is not None else 0))

    def add(self, X, q0, n, ell, power, vel_kind, vel_params, dt, mode=DIRECT, precision=FP64, t0=0.0):
        X = np.ascontiguousarray(X, dtype=np.float64)
        q = np.ascontiguousarray(np.asarray(q0, dtype=np.float64).reshape(X.shape[0], -1))
        vp = (ctypes.c_double * 4)(*(list(np.asarray(vel_params, dtype=float)) + [0.0] * 4)[:4])
        p = Problem(X.shape[0], X.ctypes.data, n, ell, float(power), mode, precision, vel_kind, vp,
                    float(t0), float(dt), q.shape[1], q.ctypes.data)
        pid = ctypes.c_int()
        _check(load().rbfsl_batch_add(self._h, ctypes.byref(p), ctypes.byref(pid)))
        self._keep[pid.value] = (X.shape[0], q.shape[1])
        return pid.value

    def remove(self, pid):
        _check(load().rbfsl_batch_remove(self._h, pid))
        self._keep.pop(pid, None)

    def step(self, nsteps=1):
        _check(load().rbfsl_batch_step(self._h, nsteps))

    def get_q(self, pid):
        N, T = self._keep[pid]
        out = np.empty((N, T))
        _check(load().rbfsl_batch_get_q(self._h, pid, out.ctypes.data))
        return out

    def stats(self, pid) -> Stats:
        s = Stats()
        _check(load().rbfsl_batch_problem_stats(self._h, pid, ctypes.byref(s)))
        return s

    def set_graph(self, use):
        _check(load().rbfsl_batch_set_graph(self._h, int(bool(use))))

    def autotune(self):
        buf = (ctypes.c_int * 96)()
        _check(load().rbfsl_batch_autotune(self._h, buf, 96))
        out = []
        for i in range(0, 96, 3):
            if buf[i] == 0:
                break
            out.append((buf[i], buf[i + 1], buf[i + 2]))
        return out

    def close(self):
        if self._h:
            load().rbfsl_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Request(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("problem", Problem), ("steps", ctypes.c_int),
                ("pu_centers", ctypes.c_void_p), ("pu_Mp", ctypes.c_int64),
                ("pu_radius", ctypes.c_double), ("pu_weight", ctypes.c_int)]


class RequestStats(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("finish_s", ctypes.c_double), ("steps", ctypes.c_int64),
                ("node_updates", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("status", ctypes.c_int), ("message", ctypes.c_char * 160),
                ("failed_points", ctypes.c_int64)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int),
                ("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("now_s", ctypes.c_double)]


class Server:
    """Serving loop with continuous batching (rbfsl_server_*)."""

    def __init__(self, device=0, budget_bytes=150 * 10 ** 9, max_slots=64):
        self._h = ctypes.c_void_p()
        self._shape = {}
        _check(load().rbfsl_server_create(ctypes.byref(self._h), device, int(budget_bytes), max_slots))

    def submit(self, X, q0, n, ell, power, vel_kind, vel_params, dt, steps, method=LOCAL,
               mode=DIRECT, precision=FP64, t0=0.0, centers=None, radius=0.0, weight=PU_WENDLAND):
        X = np.ascontiguousarray(X, dtype=np.float64)
        q = np.ascontiguousarray(np.asarray(q0, dtype=np.float64).reshape(X.shape[0], -1))
        vp = (ctypes.c_double * 4)(*(list(np.asarray(vel_params, dtype=float)) + [0.0] * 4)[:4])
        p = Problem(X.shape[0], X.ctypes.data, n, ell, float(power), mode, precision, vel_kind, vp,
                    float(t0), float(dt), q.shape[1], q.ctypes.data)
        C = None if centers is None else np.ascontiguousarray(centers, dtype=np.float64)
        r = Request(method, p, steps, None if C is None else C.ctypes.data,
                    0 if C is None else C.shape[0], float(radius), weight)
        t = ctypes.c_uint64()
        _check(load().rbfsl_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._shape[t.value] = (X.shape[0], q.shape[1])
        return t.value

    def poll(self, ticket):
        st = ctypes.c_int()
        _check(load().rbfsl_server_poll(self._h, ticket, ctypes.byref(st)))
        return st.value

    def result(self, ticket, raise_on_failure=True):
        """(field, stats) of a finished request; (None, stats) for a failed one when
        raise_on_failure is False."""
        N, T = self._shape.pop(ticket)
        out = np.empty((N, T))
        st = RequestStats()
        rc = load().rbfsl_server_result(self._h, ticket, out.ctypes.data, ctypes.byref(st))
        if rc != OK:
            if raise_on_failure:
                raise RbfslError(rc, st.message.decode() or "request failed")
            return None, st
        return out, st

    def wait_idle(self, timeout_s=600.0):
        _check(load().rbfsl_server_wait_idle(self._h, float(timeout_s)))

    def info(self) -> ServerInfo:
        i = ServerInfo()
        _check(load().rbfsl_server_info(self._h, ctypes.byref(i)))
        return i

    def close(self):
        if self._h:
            load().rbfsl_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbfsl_global_eval_tc(p, x, kernel, eps, c, out, workspace=None, status=None, stream=None):
    """Tensor-core (split TF32) evaluation; workspace: a uint8 device tensor (allocated here
    when None); status: an int32 device tensor of one element or None."""
    import torch
    T = c.shape[1] if c.dim() == 2 else 1
    need = load().rbfsl_global_eval_tc_workspace_bytes(p.shape[0], x.shape[0], T)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=c.device)
    _check(load().rbfsl_global_eval_tc(_ptr(p), p.shape[0], _ptr(x), x.shape[0], kernel, float(eps),
                                       _ptr(c), _dtype_code(c), T, _ptr(out), _ptr(workspace),
                                       workspace.numel(), _ptr(status), _stream(stream)))
    return workspace


def rbfsl_global_eval_pairs(p, x, kernel, eps, c, out, workspace=None, stream=None):
    """FP64-accurate evaluation in FP32-pair arithmetic; c: FP64 N x T; out: float32 Nq x T x 2;
    workspace: a uint8 device tensor (allocated here when None, 256-byte aligned)."""
    import torch
    T = c.shape[1] if c.dim() == 2 else 1
    need = load().rbfsl_global_eval_pairs_workspace_bytes(p.shape[0], x.shape[0], T)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=c.device)
    _check(load().rbfsl_global_eval_pairs(_ptr(p), p.shape[0], _ptr(x), x.shape[0], kernel, float(eps),
                                          _ptr(c), T, _ptr(out), _ptr(workspace), workspace.numel(),
                                          _stream(stream)))
    return workspace


def _f64_or_pairs(t):
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32 and t.dim() >= 2 and t.shape[-1] == 2:
        return F32X2
    raise TypeError(f"expected float64, or float32 pairs (last dimension 2); got {t.dtype} {tuple(t.shape)}")


def rbfsl_global_cardinal(LU, perm, x, kernel, eps, p, E, stream=None):
    """E = Phi(p, x) A_X^-1 from the factor of rbfsl_global_factor; E: (Nq, N) float64, or
    (Nq, N, 2) float32 pairs."""
    _check(load().rbfsl_global_cardinal(_ptr(LU), _ptr(perm), _ptr(x), x.shape[0], kernel, float(eps),
                                        _ptr(p), p.shape[0], _ptr(E), _f64_or_pairs(E), _stream(stream)))


def rbfsl_cardinal_apply(E, q, out, workspace=None, stream=None):
    """out = E q (FP64, or FP32-pair arithmetic for pair tensors); workspace: a uint8 device
    tensor (allocated here when None), returned for reuse."""
    import torch
    code = _f64_or_pairs(E)
    if _f64_or_pairs(q) != code or _f64_or_pairs(out) != code:
        raise TypeError("E, q and out must all be float64 or all FP32 pairs")
    fdim = 2 if code == F64 else 3
    T = q.shape[1] if q.dim() == fdim else 1
    need = load().rbfsl_cardinal_apply_workspace_bytes(E.shape[0], E.shape[1], T)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=E.device)
    _check(load().rbfsl_cardinal_apply(_ptr(E), E.shape[0], E.shape[1], _ptr(q), T, code, _ptr(out),
                                       _ptr(workspace), workspace.numel(), _stream(stream)))
    return workspace


# --------------------------------------------------------------------------- context
class Context:
    """Algorithm 1 on the device: set the problem, then step. Method names follow the C ABI
    (rbfsl_set_nodes -> set_nodes, ...)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        self.stream = _stream(stream) if stream is not None else 0
        _check(load().rbfsl_create(ctypes.byref(self._h), device, self.stream))
        self.N = 0
        self.T = 0

    def _c(self, rc):
        return _check(rc, self._h)

    def close(self):
        if self._h:
            load().rbfsl_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nodes(self, X):
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float64)
            self._c(load().rbfsl_set_nodes(self._h, X.ctypes.data, X.shape[0], HOST))
        else:
            self._c(load().rbfsl_set_nodes(self._h, _ptr(X), X.shape[0], DEVICE))
        self.N = X.shape[0]

    def set_velocity(self, kind, params):
        prm = np.ascontiguousarray(params, dtype=np.float64)
        self._c(load().rbfsl_set_velocity(self._h, kind, prm.ctypes.data, prm.size))

    def set_method(self, method, stencil_mode=DIRECT):
        self._c(load().rbfsl_set_method(self._h, method, stencil_mode))

    def set_stencil_size(self, n):
        self._c(load().rbfsl_set_stencil_size(self._h, n))

    def set_sh_degree(self, ell):
        self._c(load().rbfsl_set_sh_degree(self._h, ell))

    def set_kernel(self, kind, param):
        self._c(load().rbfsl_set_kernel(self._h, kind, float(param)))

    def set_pu(self, centers, radius=0.0, weight_kind=PU_WENDLAND):
        c = np.ascontiguousarray(centers, dtype=np.float64)
        self._c(load().rbfsl_set_pu(self._h, c.ctypes.data, c.shape[0], float(radius), weight_kind, HOST))

    def set_precision(self, prec):
        self._c(load().rbfsl_set_precision(self._h, prec))

    def set_dt(self, dt):
        self._c(load().rbfsl_set_dt(self._h, float(dt)))

    def set_integrator(self, order):
        self._c(load().rbfsl_set_integrator(self._h, order))

    def set_global_form(self, form):
        self._c(load().rbfsl_set_global_form(self._h, form))

    def set_global_eval(self, kind):
        self._c(load().rbfsl_set_global_eval(self._h, kind))

    def set_time(self, t):
        self._c(load().rbfsl_set_time(self._h, float(t)))

    def set_tracers(self, q):
        if isinstance(q, np.ndarray):
            q2 = np.ascontiguousarray(q.reshape(q.shape[0], -1))
            code = F64 if q2.dtype == np.float64 else F32
            if q2.dtype not in (np.float64, np.float32):
                q2 = q2.astype(np.float64); code = F64
            self._c(load().rbfsl_set_tracers(self._h, q2.ctypes.data, q2.shape[0], q2.shape[1], code, HOST))
            self.T = q2.shape[1]
        else:
            q2 = q.reshape(q.shape[0], -1)
            dev = DEVICE if q2.is_cuda else HOST
            self._c(load().rbfsl_set_tracers(self._h, _ptr(q2), q2.shape[0], q2.shape[1],
                                             _dtype_code(q2), dev))
            self.T = q2.shape[1]

    def step(self, nsteps=1):
        self._c(load().rbfsl_step(self._h, nsteps))

    def get_q(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty((self.N, self.T), dtype=dtype)
        if isinstance(out, np.ndarray):
            code = F64 if out.dtype == np.float64 else F32
            self._c(load().rbfsl_get_q(self._h, out.ctypes.data, code, HOST))
        else:
            self._c(load().rbfsl_get_q(self._h, _ptr(out), _dtype_code(out),
                                       DEVICE if out.is_cuda else HOST))
        return out

    def get_stats(self) -> Stats:
        s = Stats()
        self._c(load().rbfsl_get_stats(self._h, ctypes.byref(s)))
        return s

    def last_step_buffers(self):
        xi, idx, w = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._c(load().rbfsl_last_step_buffers(self._h, ctypes.byref(xi), ctypes.byref(idx), ctypes.byref(w)))
        return xi.value, idx.value, w.value

    def last_step_tensors(self, n, weights_dtype):
        """Copies of the last step's departure points (N x 3), stencils (N x n) and weights as
        torch tensors: N x n float64 (weights_dtype float64, the FP64 step) or N x n x 2 float32
        FP32 pairs (weights_dtype float32, the mixed-precision step)."""
        import torch
        xi, idx, w = self.last_step_buffers()
        torch.cuda.synchronize()
        wt, wshape = ("<f8", (self.N, n)) if weights_dtype == torch.float64 else ("<f4", (self.N, n, 2))
        out = []
        for ptr, shape, ts in ((xi, (self.N, 3), "<f8"), (idx, (self.N, n), "<i4"), (w, wshape, wt)):
            out.append(None if not ptr else torch.as_tensor(_DeviceView(ptr, shape, ts), device="cuda").clone())
        return tuple(out)


class _DeviceView:
    """Exposes a library-owned device buffer through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "strides": None, "version": 3}

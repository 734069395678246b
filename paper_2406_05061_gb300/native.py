"""Thin ctypes binding of libprogot.so (include/progot.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. Device arrays are torch CUDA tensors (float32, contiguous); their raw
pointers and torch's current stream are handed to the C ABI. There is no CPU
fallback: if the library is not built or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprogot.so")

PROGOT_OK = 0
PROGOT_ERR_INVALID_ARG = 1
PROGOT_ERR_NOT_CONVERGED = 2
PROGOT_ERR_NUMERIC = 3
PROGOT_ERR_OOM = 4
PROGOT_ERR_CUDA = 5
PROGOT_ERR_TIMEOUT = 6
PROGOT_ERR_WORKSPACE = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_CONVERGED", 3: "NUMERIC", 4: "OOM", 5: "CUDA", 6: "TIMEOUT",
                7: "WORKSPACE"}

PRECISIONS = {"fp32": 0, "bf16x3": 1, "bf16": 2}
ALPHA_KINDS = {"constant": 0, "accelerated": 1, "decelerated": 2}

# (name, restype, argtypes) of every exported symbol of include/progot.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_SZ = ctypes.c_size_t
SIGNATURES = [
    ("progot_last_error_string", ctypes.c_char_p, []),
    ("progot_version", ctypes.c_char_p, []),
    ("progot_workspace_size", _SZ, [_I64, _I64, _I32, _I32]),
    ("sinkhorn_potentials", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _D, _D, _I32, _I32, _P, _P, _I32, _P, _P, _P, _SZ, _P]),
    ("entropic_map_apply", ctypes.c_int, [_P, _I64, _P, _I64, _I32, _I32, _P, _P, _P, _I32, _P, _P, _SZ, _P]),
    ("coupling_marginals", ctypes.c_int,
     [_P, _I64, _P, _I64, _I32, _P, _P, _D, _I32, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("coupling_marginals_noalloc", ctypes.c_int,
     [_P, _I64, _P, _I64, _I32, _P, _P, _D, _I32, _P, _P, _P, _P, _P, _P]),
    ("progot_solve", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _I32, _P, _P, _P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("progot_schedule_alpha", ctypes.c_int, [_I32, _I32, _P]),
    ("progot_mean_cost", ctypes.c_int, [_P, _I64, _P, _I64, _I32, _P, _P, _SZ, _P]),
    ("progot_schedule_eps", ctypes.c_int,
     [_P, _I64, _P, _P, _I64, _P, _I64, _I32, _I32, _P, _P, _I32, _D, _D, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    ("progot_set_stall_window", ctypes.c_int, [_I32]),
    ("progot_set_map_tc", ctypes.c_int, [_I32]),
    ("progot_set_loop_tc", ctypes.c_int, [_I32]),
    ("progot_set_wait_limit_ns", ctypes.c_int, [ctypes.c_uint64]),
    ("progot_test_withhold_initial_betas", ctypes.c_int, [_I32]),
    ("progot_launch_count", ctypes.c_int64, [_I32]),
    ("progot_batched_workspace_size", _SZ, [_P, _I32, _I32, _I32]),
    ("progot_solve_batched", ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _P, _SZ, _P]),
    ("progot_set_batch_engine", ctypes.c_int, [_I32]),
    ("progot_batch_plan_workspace_size", _SZ, [_P, _I32, _I32]),
    ("progot_batch_plan_create", ctypes.c_int, [_P, _I32, _I32, _I32, _P, _SZ, _P]),
    ("progot_batch_plan_run", ctypes.c_int, [_P, _I32, _P]),
    ("progot_batch_plan_collect", ctypes.c_int, [_P, _P, _P]),
    ("progot_batch_plan_set_target", ctypes.c_int, [_P, _I32]),
    ("progot_batch_plan_autotune", ctypes.c_int, [_P, _P, _P, _P]),
    ("progot_batch_plan_destroy", None, [_P]),
    ("progot_server_create", ctypes.c_void_p, [_SZ, _I32, _I32, _I32]),
    ("progot_server_submit", ctypes.c_int64, [_P, _P]),
    ("progot_server_wait", ctypes.c_int, [_P, _I64, _P]),
    ("progot_server_stats", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("progot_server_destroy", None, [_P]),
    ("progot_schedule_tau", ctypes.c_int, [_I32, _D, _D, _P]),
    ("progot_solve_theta", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _I32, _P, _D, _P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("coupling_metrics", ctypes.c_int, [_P, _P, _I64, _P, _P, _I64, _I32, _P, _P, _P, _D, _P, _P, _SZ, _P]),
    ("sinkhorn_divergence", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _D, _D, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    ("coupling_diagonal", ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _D, _P, _P, _P, _P, _SZ, _P]),
    ("sinkhorn_potentials_pnorm", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _D, _D, _D, _I32, _P, _P, _I32, _P, _P, _P, _SZ, _P]),
    ("progot_solve_pnorm", ctypes.c_int,
     [_P, _P, _I64, _P, _P, _I64, _I32, _D, _I32, _P, _P, _D, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("entropic_map_apply_pnorm", ctypes.c_int, [_P, _I64, _P, _I64, _I32, _D, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
    ("coupling_metrics_pnorm", ctypes.c_int, [_P, _P, _I64, _P, _P, _I64, _I32, _D, _P, _P, _P, _D, _P, _P, _SZ, _P]),
    ("progot_mean_cost_pnorm", ctypes.c_int, [_P, _I64, _P, _I64, _I32, _D, _P, _P, _SZ, _P]),
    ("progot_profile", ctypes.c_int, [_I32]),
    ("progot_profile_read", ctypes.c_int, [_I32, _P, _P, _P, _P]),
]

_lib = None


class ProgOTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libprogot.so (built in-tree by paper_2406_05061_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2406_05061_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().progot_last_error_string().decode()


def _check(rc: int, allow_not_converged: bool = True) -> int:
    if rc == PROGOT_OK or (allow_not_converged and rc == PROGOT_ERR_NOT_CONVERGED):
        return rc
    raise ProgOTError(rc, last_error())


# ------------------------------------------------------------------ helpers
def _torch():
    import torch  # noqa: PLC0415  (imported lazily: the CPU tests only load the library)
    return torch


def _dev(t, name, shape=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _opt(t, name, shape=None):
    return None if t is None else _dev(t, name, shape)


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prec(precision) -> int:
    if isinstance(precision, int):
        return precision
    return PRECISIONS[precision]


def workspace_size(n: int, m: int, d: int, precision="fp32") -> int:
    return int(lib().progot_workspace_size(n, m, d, _prec(precision)))


class Workspace:
    """A reusable device workspace (torch uint8 buffer, 256-byte aligned)."""

    def __init__(self, n: int, m: int, d: int, precision="fp32", device=None):
        torch = _torch()
        self.bytes = workspace_size(n, m, d, precision)
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.ptr = (base + 255) & ~255
        self.dims = (n, m, d, _prec(precision))

    def covers(self, n, m, d, precision) -> bool:
        return workspace_size(n, m, d, precision) <= self.bytes


def _ws(ws, n, m, d, precision):
    if ws is None or not ws.covers(n, m, d, precision):
        ws = Workspace(n, m, d, precision)
    return ws


def _host_f64(v, k=None):
    arr = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    if k is not None and arr.shape != (k,):
        raise ValueError(f"expected {k} values, got shape {arr.shape}")
    return arr


def _hp(arr):
    return arr.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ API
@dataclass
class SinkhornOut:
    f: object
    g: object
    iters: int
    err: float
    status: int


def sinkhorn_potentials(x, y, eps, tau, max_iter=10000, a=None, b=None, f=None, g=None, precision="fp32",
                        workspace=None, stream=None) -> SinkhornOut:
    """Alg. 1 on the GPU. f, g (CUDA float32) are used as the initial potentials when
    given (and overwritten), else zero-initialised tensors are returned."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    init_zero = 1 if (f is None and g is None) else 0
    if f is None:
        f = torch.zeros(n, dtype=torch.float32, device=x.device)
    if g is None:
        g = torch.zeros(m, dtype=torch.float32, device=x.device)
    ws = _ws(workspace, n, m, d, precision)
    it = ctypes.c_int32(0)
    err = ctypes.c_double(0.0)
    rc = lib().sinkhorn_potentials(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                   float(eps), float(tau), int(max_iter), _prec(precision), _dev(f, "f", (n,)),
                                   _dev(g, "g", (m,)), init_zero, ctypes.byref(it), ctypes.byref(err),
                                   ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc)
    return SinkhornOut(f, g, it.value, err.value, rc)


def entropic_map_apply(xq, y, g_all, eps, alpha, precision="fp32", out=None, workspace=None, stream=None):
    """Alg. 3 (the progressive map) on nq query points; returns out (nq x d)."""
    torch = _torch()
    _dev(xq, "xq"), _dev(y, "y")
    nq, d = xq.shape
    m = y.shape[0]
    K = g_all.shape[0] if g_all.dim() == 2 else 1
    eps_h = _host_f64(eps, K)
    al_h = _host_f64(alpha, K)
    if out is None:
        out = torch.empty_like(xq)
    ws = _ws(workspace, nq, m, d, precision)
    rc = lib().entropic_map_apply(_dev(xq, "xq"), nq, _dev(y, "y"), m, d, K, _dev(g_all.contiguous(), "g_all"),
                                  _hp(eps_h), _hp(al_h), _prec(precision), _dev(out, "out", (nq, d)),
                                  ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return out


def coupling_marginals(x, y, f, g, eps, a=None, b=None, precision="fp32", workspace=None, stream=None):
    """Row and column sums of P = exp((f (+) g - C)/eps) and ||r - a||_1 + ||c - b||_1."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    row = torch.empty(n, dtype=torch.float32, device=x.device)
    col = torch.empty(m, dtype=torch.float32, device=x.device)
    err = ctypes.c_double(0.0)
    ws = _ws(workspace, n, m, d, precision)
    rc = lib().coupling_marginals(_dev(x, "x"), n, _dev(y, "y"), m, d, _dev(f, "f", (n,)), _dev(g, "g", (m,)),
                                  float(eps), _prec(precision), _dev(row, "row"), _dev(col, "col"),
                                  _opt(a, "a", (n,)), _opt(b, "b", (m,)), ctypes.byref(err),
                                  ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return row, col, err.value


@dataclass
class ProgOTOut:
    x_out: object
    g_all: object
    f_last: object
    x_last: object
    iters: list
    errs: list
    status: int


def progot_solve(x, y, alpha, eps, tau, max_iter=10000, a=None, b=None, precision="fp32", workspace=None,
                 stream=None, out=None) -> ProgOTOut:
    """Alg. 2 on the GPU: K = len(eps) warm-started Sinkhorn solves and displacements."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    K = len(eps)
    al_h, eps_h, tau_h = _host_f64(alpha, K), _host_f64(eps, K), _host_f64(tau, K)
    if out is None:
        out = dict(x_out=torch.empty_like(x), g_all=torch.empty((K, m), dtype=torch.float32, device=x.device),
                   f_last=torch.empty(n, dtype=torch.float32, device=x.device), x_last=torch.empty_like(x))
    iters = np.zeros(K, dtype=np.int32)
    errs = np.zeros(K, dtype=np.float64)
    ws = _ws(workspace, n, m, d, precision)
    rc = lib().progot_solve(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d, K,
                            _hp(al_h), _hp(eps_h), _hp(tau_h), int(max_iter), _prec(precision),
                            _dev(out["x_out"], "x_out", (n, d)), _dev(out["g_all"], "g_all", (K, m)),
                            _opt(out.get("f_last"), "f_last", (n,)), _opt(out.get("x_last"), "x_last", (n, d)),
                            _hp(iters), _hp(errs), ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc)
    return ProgOTOut(out["x_out"], out["g_all"], out.get("f_last"), out.get("x_last"), iters.tolist(),
                     errs.tolist(), rc)


def progot_solve_theta(x, y, alpha, theta, tau, max_iter=10000, a=None, b=None, precision="fp32", workspace=None,
                       stream=None, out=None):
    """Alg. 2 with eps_k = theta * mean cost(X^(k), Y) / 20 (Sec. 5.2); K = len(alpha).
    Returns (ProgOTOut, eps_k array)."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    K = len(alpha)
    al_h, tau_h = _host_f64(alpha, K), _host_f64(tau, K)
    if out is None:
        out = dict(x_out=torch.empty_like(x), g_all=torch.empty((K, m), dtype=torch.float32, device=x.device),
                   f_last=torch.empty(n, dtype=torch.float32, device=x.device), x_last=torch.empty_like(x))
    iters = np.zeros(K, dtype=np.int32)
    errs = np.zeros(K, dtype=np.float64)
    eps_out = np.zeros(K, dtype=np.float64)
    ws = _ws(workspace, n, m, d, precision)
    rc = lib().progot_solve_theta(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d, K,
                                  _hp(al_h), float(theta), _hp(tau_h), int(max_iter), _prec(precision),
                                  _dev(out["x_out"], "x_out", (n, d)), _dev(out["g_all"], "g_all", (K, m)),
                                  _opt(out.get("f_last"), "f_last", (n,)), _opt(out.get("x_last"), "x_last", (n, d)),
                                  _hp(iters), _hp(errs), _hp(eps_out), ctypes.c_void_p(ws.ptr), ws.bytes,
                                  _stream(stream))
    _check(rc)
    return (ProgOTOut(out["x_out"], out["g_all"], out.get("f_last"), out.get("x_last"), iters.tolist(),
                      errs.tolist(), rc), eps_out)


def progot_schedule_tau(K: int, tau_first: float, tau_last: float) -> np.ndarray:
    out = np.zeros(K, dtype=np.float64)
    _check(lib().progot_schedule_tau(int(K), float(tau_first), float(tau_last), _hp(out)), allow_not_converged=False)
    return out


class CouplingMetricsStruct(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("transport_cost", "entropy", "dual", "mass", "err_row", "err_col")]


def coupling_metrics(x, y, f, g, eps, a=None, b=None, x_cost=None, workspace=None, stream=None) -> dict:
    """<P, C>, E(P), the eq. (5) objective, sum P and both marginal errors (Sec. 5.2);
    with x_cost the transport cost integrates ||xc_i - y_j||^2 against P (on x)."""
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    ws = _ws(workspace, n, m, d, "fp32")
    res = CouplingMetricsStruct()
    rc = lib().coupling_metrics(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                _dev(f, "f", (n,)), _dev(g, "g", (m,)), _opt(x_cost, "x_cost", (n, d)), float(eps),
                                ctypes.byref(res),
                                ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return {k: getattr(res, k) for k, _ in CouplingMetricsStruct._fields_}


def sinkhorn_divergence(x, y, eps, tau, max_iter=10000, a=None, b=None, precision="fp32", workspace=None,
                        stream=None):
    """D_eps(X, Y) of eq. (8). Returns (D, [OT_xy, OT_xx, OT_yy], [iters ...], status)."""
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    k = max(n, m)
    ws = _ws(workspace, k, k, d, precision)
    val = ctypes.c_double(0.0)
    parts = np.zeros(3, dtype=np.float64)
    its = np.zeros(3, dtype=np.int32)
    rc = lib().sinkhorn_divergence(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                   float(eps), float(tau), int(max_iter), _prec(precision), ctypes.byref(val),
                                   _hp(parts), _hp(its), ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc)
    return val.value, parts.tolist(), its.tolist(), rc


def coupling_diagonal(x, y, f, g, eps, log_diag=None, workspace=None, stream=None):
    """Tr(P) and KL(Id/n || P) for n = m (Sec. 5.3, Prop. 3). Returns (trace, kl)."""
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    if y.shape != x.shape:
        raise ValueError("coupling_diagonal needs x and y of the same shape")
    ws = _ws(workspace, n, n, d, "fp32")
    tr = ctypes.c_double(0.0)
    kl = ctypes.c_double(0.0)
    rc = lib().coupling_diagonal(_dev(x, "x"), _dev(y, "y"), n, d, _dev(f, "f", (n,)), _dev(g, "g", (n,)),
                                 float(eps), _opt(log_diag, "log_diag", (n,)), ctypes.byref(tr), ctypes.byref(kl),
                                 ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return tr.value, kl.value


# ------------------------------------------------------- p-norm cost (Sec. 5.2)
def sinkhorn_potentials_pnorm(x, y, p, eps, tau, max_iter=10000, a=None, b=None, f=None, g=None, workspace=None,
                              stream=None) -> SinkhornOut:
    """Alg. 1 for the cost h(x - y) = (1/p) sum_k |x_k - y_k|^p (float32 CUDA cores)."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    init_zero = 1 if (f is None and g is None) else 0
    if f is None:
        f = torch.zeros(n, dtype=torch.float32, device=x.device)
    if g is None:
        g = torch.zeros(m, dtype=torch.float32, device=x.device)
    ws = _ws(workspace, n, m, d, "fp32")
    it = ctypes.c_int32(0)
    err = ctypes.c_double(0.0)
    rc = lib().sinkhorn_potentials_pnorm(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                         float(p), float(eps), float(tau), int(max_iter), _dev(f, "f", (n,)),
                                         _dev(g, "g", (m,)), init_zero, ctypes.byref(it), ctypes.byref(err),
                                         ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc)
    return SinkhornOut(f, g, it.value, err.value, rc)


def progot_solve_pnorm(x, y, p, alpha, tau, eps=None, theta=None, max_iter=10000, a=None, b=None, workspace=None,
                       stream=None, out=None):
    """Alg. 2 for the p-norm cost with an eps schedule, or the theta rule when eps is None.
    Returns (ProgOTOut, eps_k array)."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    K = len(alpha)
    al_h, tau_h = _host_f64(alpha, K), _host_f64(tau, K)
    eps_h = None if eps is None else _host_f64(eps, K)
    if eps_h is None and theta is None:
        raise ValueError("give eps or theta")
    if out is None:
        out = dict(x_out=torch.empty_like(x), g_all=torch.empty((K, m), dtype=torch.float32, device=x.device),
                   f_last=torch.empty(n, dtype=torch.float32, device=x.device), x_last=torch.empty_like(x))
    iters = np.zeros(K, dtype=np.int32)
    errs = np.zeros(K, dtype=np.float64)
    eps_out = np.zeros(K, dtype=np.float64)
    ws = _ws(workspace, n, m, d, "fp32")
    rc = lib().progot_solve_pnorm(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                  float(p), K, _hp(al_h), None if eps_h is None else _hp(eps_h),
                                  float(theta or 0.0), _hp(tau_h), int(max_iter), _dev(out["x_out"], "x_out", (n, d)),
                                  _dev(out["g_all"], "g_all", (K, m)), _opt(out.get("f_last"), "f_last", (n,)),
                                  _opt(out.get("x_last"), "x_last", (n, d)), _hp(iters), _hp(errs), _hp(eps_out),
                                  ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc)
    return (ProgOTOut(out["x_out"], out["g_all"], out.get("f_last"), out.get("x_last"), iters.tolist(),
                      errs.tolist(), rc), eps_out)


def entropic_map_apply_pnorm(xq, y, p, g_all, eps, alpha, out=None, workspace=None, stream=None):
    """Alg. 3 for the p-norm cost; returns out (nq x d)."""
    torch = _torch()
    _dev(xq, "xq"), _dev(y, "y")
    nq, d = xq.shape
    m = y.shape[0]
    K = g_all.shape[0] if g_all.dim() == 2 else 1
    eps_h, al_h = _host_f64(eps, K), _host_f64(alpha, K)
    if out is None:
        out = torch.empty_like(xq)
    ws = _ws(workspace, nq, m, d, "fp32")
    rc = lib().entropic_map_apply_pnorm(_dev(xq, "xq"), nq, _dev(y, "y"), m, d, float(p), K,
                                        _dev(g_all.contiguous(), "g_all"), _hp(eps_h), _hp(al_h),
                                        _dev(out, "out", (nq, d)), ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return out


def coupling_metrics_pnorm(x, y, p, f, g, eps, a=None, b=None, x_cost=None, workspace=None, stream=None) -> dict:
    """coupling_metrics for the p-norm cost."""
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    ws = _ws(workspace, n, m, d, "fp32")
    res = CouplingMetricsStruct()
    rc = lib().coupling_metrics_pnorm(_dev(x, "x"), _opt(a, "a", (n,)), n, _dev(y, "y"), _opt(b, "b", (m,)), m, d,
                                      float(p), _dev(f, "f", (n,)), _dev(g, "g", (m,)), _opt(x_cost, "x_cost", (n, d)),
                                      float(eps), ctypes.byref(res),
                                      ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream))
    _check(rc, allow_not_converged=False)
    return {k: getattr(res, k) for k, _ in CouplingMetricsStruct._fields_}


def progot_mean_cost_pnorm(x, y, p, workspace=None, stream=None) -> float:
    n, d = x.shape
    m = y.shape[0]
    ws = _ws(workspace, n, m, d, "fp32")
    out = ctypes.c_double(0.0)
    _check(lib().progot_mean_cost_pnorm(_dev(x, "x"), n, _dev(y, "y"), m, d, float(p), ctypes.byref(out),
                                        ctypes.c_void_p(ws.ptr), ws.bytes, _stream(stream)), allow_not_converged=False)
    return out.value


def progot_schedule_alpha(K: int, kind="constant") -> np.ndarray:
    out = np.zeros(K, dtype=np.float64)
    _check(lib().progot_schedule_alpha(int(K), ALPHA_KINDS[kind] if isinstance(kind, str) else int(kind), _hp(out)),
           allow_not_converged=False)
    return out


def progot_mean_cost(x, y, workspace=None, stream=None) -> float:
    n, d = x.shape
    m = y.shape[0]
    ws = _ws(workspace, n, m, d, "fp32")
    out = ctypes.c_double(0.0)
    _check(lib().progot_mean_cost(_dev(x, "x"), n, _dev(y, "y"), m, d, ctypes.byref(out), ctypes.c_void_p(ws.ptr),
                                  ws.bytes, _stream(stream)), allow_not_converged=False)
    return out.value


def progot_schedule_eps(x, y, y_test, alpha, s_grid=None, beta0=5.0, tau=1e-6, max_iter=10000, b=None,
                        precision="fp32", workspace=None, stream=None):
    """Alg. 4 on the GPU; returns (eps_k array, scores per s_p, p_star)."""
    n, d = x.shape
    m = y.shape[0]
    mt = y_test.shape[0]
    if s_grid is None:
        s_grid = [2.0 ** e for e in range(-3, 4)]
    K = len(alpha)
    al_h, sg_h = _host_f64(alpha, K), _host_f64(s_grid)
    P = sg_h.shape[0]
    eps_out = np.zeros(K)
    errors = np.zeros(P)
    pstar = ctypes.c_int32(0)
    nmax = max(n, m, mt)
    ws = _ws(workspace, nmax, nmax, d, precision)
    _check(lib().progot_schedule_eps(_dev(x, "x"), n, _dev(y, "y"), _opt(b, "b", (m,)), m,
                                     _dev(y_test, "y_test", (mt, d)), mt, d, K, _hp(al_h), _hp(sg_h), P,
                                     float(beta0), float(tau), int(max_iter), _prec(precision), _hp(eps_out),
                                     _hp(errors), ctypes.byref(pstar), ctypes.c_void_p(ws.ptr), ws.bytes,
                                     _stream(stream)), allow_not_converged=False)
    return eps_out, errors, pstar.value


def set_map_tc(on: bool) -> None:
    """Map step of the tensor-core paths (d <= 64) on tcgen05 (True, default) or with a
    float32 CUDA-core P Y (False)."""
    _check(lib().progot_set_map_tc(1 if on else 0), allow_not_converged=False)


def set_loop_tc(on: bool) -> None:
    """Sinkhorn loops of the tensor-core paths as one persistent launch (True, default)
    or one launch per update (False)."""
    _check(lib().progot_set_loop_tc(1 if on else 0), allow_not_converged=False)


def set_wait_limit_ns(ns: int) -> None:
    """Bounded-wait limit of the persistent Sinkhorn loop in ns (0: the 2 s default)."""
    _check(lib().progot_set_wait_limit_ns(int(ns)), allow_not_converged=False)


def test_withhold_initial_betas(on: bool) -> None:
    """Test hook: persistent Sinkhorn loops start without g's initial betas, so their
    bounded wait expires (PROGOT_ERR_TIMEOUT)."""
    _check(lib().progot_test_withhold_initial_betas(1 if on else 0), allow_not_converged=False)


def set_stall_window(iters: int) -> None:
    _check(lib().progot_set_stall_window(int(iters)), allow_not_converged=False)


def launch_count(reset: bool = False) -> int:
    return int(lib().progot_launch_count(1 if reset else 0))


KERNEL_IDS = {"lse_sweep": 0, "map_sweep": 1}


def profile(enable, period: int = 1) -> None:
    """Start (True; events around every period-th launch) or stop (False) per-kernel
    CUDA-event timing inside the library."""
    _check(lib().progot_profile(max(1, int(period)) if enable else 0), allow_not_converged=False)


def profile_read(kernel: str) -> dict:
    """launches/ms/pairs of the sampled launches, worked = launches that did work."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    pairs = ctypes.c_double(0.0)
    worked = ctypes.c_int64(0)
    _check(lib().progot_profile_read(KERNEL_IDS[kernel], ctypes.byref(n), ctypes.byref(ms), ctypes.byref(pairs),
                                     ctypes.byref(worked)), allow_not_converged=False)
    return dict(launches=n.value, ms=ms.value, pairs=pairs.value, worked=worked.value)


NOALLOC_MAX_POINTS = 65536


def coupling_marginals_noalloc(x, y, f, g, eps, a=None, b=None, precision="fp32", row=None, col=None,
                               stream=None, want_err=True):
    """coupling_marginals through the allocation-free entry point: the library uses its
    own static device scratch (n, m <= 65536); the caller supplies inputs and outputs.
    With want_err=False no error is requested (NULL) and the call stays asynchronous;
    the returned error is then None."""
    torch = _torch()
    _dev(x, "x"), _dev(y, "y")
    n, d = x.shape
    m = y.shape[0]
    if row is None:
        row = torch.empty(n, dtype=torch.float32, device=x.device)
    if col is None:
        col = torch.empty(m, dtype=torch.float32, device=x.device)
    err = ctypes.c_double(0.0)
    rc = lib().coupling_marginals_noalloc(_dev(x, "x"), n, _dev(y, "y"), m, d, _dev(f, "f", (n,)),
                                          _dev(g, "g", (m,)), float(eps), _prec(precision), _dev(row, "row", (n,)),
                                          _dev(col, "col", (m,)), _opt(a, "a", (n,)), _opt(b, "b", (m,)),
                                          ctypes.byref(err) if want_err else None, _stream(stream))
    _check(rc, allow_not_converged=False)
    return row, col, (err.value if want_err else None)


class ProblemStruct(ctypes.Structure):
    """ctypes mirror of progot_problem (include/progot.h)."""
    _fields_ = [("x", _P), ("a", _P), ("n", _I64), ("y", _P), ("b", _P), ("m", _I64), ("d", _I32), ("K", _I32),
                ("alpha", _P), ("eps", _P), ("tau", _P), ("x_out", _P), ("g_all", _P), ("f_last", _P),
                ("iters", _P), ("errs", _P), ("status", _I32)]


def _problem_struct(x, y, alpha, eps, tau, x_out, g_all, f_last=None, a=None, b=None, keep=None):
    """Fill a ProblemStruct from torch CUDA tensors (batched) or numpy arrays (server)."""
    def ptr(t):
        if t is None:
            return None
        if isinstance(t, np.ndarray):
            return t.ctypes.data_as(ctypes.c_void_p)
        return ctypes.c_void_p(t.data_ptr())
    K = len(eps)
    al_h, eps_h, tau_h = _host_f64(alpha, K), _host_f64(eps, K), _host_f64(tau, K)
    iters = np.zeros(K, dtype=np.int32)
    errs = np.zeros(K, dtype=np.float64)
    n, d = x.shape
    m = y.shape[0]
    s = ProblemStruct(ptr(x), ptr(a), n, ptr(y), ptr(b), m, d, K, _hp(al_h), _hp(eps_h), _hp(tau_h), ptr(x_out),
                      ptr(g_all), ptr(f_last), _hp(iters), _hp(errs), 0)
    holder = dict(al=al_h, eps=eps_h, tau=tau_h, iters=iters, errs=errs, x=x, y=y, x_out=x_out, g_all=g_all,
                  f_last=f_last, a=a, b=b)
    if keep is not None:
        keep.append(holder)
    return s, holder


def _batch_structs(problems):
    """ProblemStruct array and output holders for a list of problem dicts (CUDA tensors)."""
    torch = _torch()
    keep = []
    arr = (ProblemStruct * len(problems))()
    outs = []
    for i, pr in enumerate(problems):
        x, y = pr["x"], pr["y"]
        _dev(x, "x"), _dev(y, "y")
        K = len(pr["eps"])
        x_out = torch.empty_like(x)
        g_all = torch.empty((K, y.shape[0]), dtype=torch.float32, device=x.device)
        f_last = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        arr[i], holder = _problem_struct(x, y, pr["alpha"], pr["eps"], pr["tau"], x_out, g_all, f_last,
                                         pr.get("a"), pr.get("b"), keep)
        outs.append(holder)
    return arr, outs


def _batch_results(arr, outs):
    return [dict(x_out=h["x_out"], g_all=h["g_all"], f_last=h["f_last"], iters=h["iters"].tolist(),
                 errs=h["errs"].tolist(), status=int(arr[i].status)) for i, h in enumerate(outs)]


def set_batch_engine(engine: str):
    """'persistent' (one launch over the batch, the default) or 'streams' (per-problem solves)."""
    _check(lib().progot_set_batch_engine({"streams": 0, "persistent": 1}[engine]))


def progot_solve_batched(problems, max_iter=10000, precision="bf16x3", n_streams=8, stream=None):
    """Solve a list of problems (dicts with x, y CUDA tensors and alpha, eps, tau) together.

    Returns a list of dicts with x_out, g_all, f_last, iters, errs, status per problem."""
    torch = _torch()
    arr, outs = _batch_structs(problems)
    L = lib()
    pc = _prec(precision)
    ws_bytes = int(L.progot_batched_workspace_size(arr, len(problems), pc, n_streams))
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
    rc = L.progot_solve_batched(arr, len(problems), int(max_iter), pc, int(n_streams), ctypes.c_void_p(ws.data_ptr()),
                                ws_bytes + 256, _stream(stream))
    _check(rc)
    return _batch_results(arr, outs)


class BatchPlan:
    """A batch of problems prepared once for repeated persistent solves (progot_batch_plan_*
    in include/progot.h): run() enqueues one solve of the whole batch (a CUDA graph replay
    by default), collect() waits and returns the per-problem results."""

    def __init__(self, problems, max_iter=10000, precision="bf16x3"):
        torch = _torch()
        self._arr, self._outs = _batch_structs(problems)
        L = lib()
        pc = _prec(precision)
        n = len(problems)
        ws_bytes = int(L.progot_batch_plan_workspace_size(self._arr, n, pc))
        self._ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(L.progot_batch_plan_create(self._arr, n, int(max_iter), pc, ctypes.c_void_p(self._ws.data_ptr()),
                                          ws_bytes + 256, ctypes.byref(h)))
        self._h = h

    def run(self, graph=True, stream=None):
        _check(lib().progot_batch_plan_run(self._h, 1 if graph else 0, _stream(stream)))

    def collect(self, stream=None, check=True):
        rc = int(lib().progot_batch_plan_collect(self._h, self._arr, _stream(stream)))
        if check:
            _check(rc)
        return _batch_results(self._arr, self._outs)

    def set_target(self, target: int):
        _check(lib().progot_batch_plan_set_target(self._h, int(target)))

    def autotune(self, stream=None):
        """Time complete runs for each segmentation target; keep and return the fastest (target, ms)."""
        t = ctypes.c_int32(0)
        ms = ctypes.c_double(0.0)
        _check(lib().progot_batch_plan_autotune(self._h, ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
        return int(t.value), float(ms.value)

    def close(self):
        if self._h:
            lib().progot_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching ProgOT server (progot_server_* in include/progot.h)."""

    def __init__(self, budget_bytes: int, n_workers: int = 8, precision="bf16x3", max_iter: int = 10000):
        L = lib()
        h = L.progot_server_create(int(budget_bytes), int(n_workers), _prec(precision), int(max_iter))
        if not h:
            raise ProgOTError(PROGOT_ERR_CUDA, last_error())
        self._h = ctypes.c_void_p(h)
        self._pending = {}

    def submit(self, x, y, alpha, eps, tau, a=None, b=None) -> int:
        """Queue one request on host arrays (float32, C-contiguous); returns its id."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        K = len(eps)
        x_out = np.empty_like(x)
        g_all = np.empty((K, y.shape[0]), dtype=np.float32)
        f_last = np.empty(x.shape[0], dtype=np.float32)
        st, holder = _problem_struct(x, y, alpha, eps, tau, x_out, g_all, f_last,
                                     None if a is None else np.ascontiguousarray(a, dtype=np.float32),
                                     None if b is None else np.ascontiguousarray(b, dtype=np.float32))
        holder["struct"] = st
        rid = int(lib().progot_server_submit(self._h, ctypes.byref(st)))
        if rid < 0:
            raise ProgOTError(-rid, last_error())
        self._pending[rid] = holder
        return rid

    def wait(self, rid: int) -> dict:
        lat = ctypes.c_double(0.0)
        rc = int(lib().progot_server_wait(self._h, int(rid), ctypes.byref(lat)))
        h = self._pending.pop(rid)
        return dict(status=rc, latency_ms=lat.value, x_out=h["x_out"], g_all=h["g_all"], f_last=h["f_last"],
                    iters=h["iters"].tolist(), errs=h["errs"].tolist())

    def stats(self) -> dict:
        c, f = ctypes.c_int64(0), ctypes.c_int64(0)
        u, pk = ctypes.c_size_t(0), ctypes.c_size_t(0)
        lib().progot_server_stats(self._h, ctypes.byref(c), ctypes.byref(f), ctypes.byref(u), ctypes.byref(pk))
        return dict(completed=c.value, in_flight=f.value, bytes_in_use=u.value, peak_bytes=pk.value)

    def close(self):
        if self._h:
            lib().progot_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""GOAT (graph matching via optimal transport) on GB300: thin Python binding of libgoat.

Every function here marshals torch CUDA tensors into the C ABI declared in
``include/goat.h`` and calls it; all arithmetic runs in libgoat's sm_103a
kernels.  There is no CPU fallback: if ``libgoat.so`` is missing or the device
is not sm_103, the calls raise.

Names follow the C ABI: ``goat_match``, ``goat_gradient``, ``goat_sinkhorn``,
``goat_line_search``, ``goat_fw_update``, ``goat_project``, ``goat_objective``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgoat.so")

GOAT_OK = 0
GOAT_ERR_INVALID_ARG = -1
GOAT_ERR_NOT_CONVERGED = -2
GOAT_ERR_CUDA = -3
GOAT_ERR_OUT_OF_MEMORY = -4
GOAT_ERR_NAN = -5
GOAT_ERR_TIMEOUT = -6
GOAT_ERR_UNSUPPORTED = -7

GOAT_DTYPE_U8 = 0
GOAT_DTYPE_F32 = 1
GOAT_PREC_BF16 = 0
GOAT_PREC_FP32 = 1
GOAT_PREC_FP8 = 2
GOAT_PREC_BF16_SPLIT = 3
GOAT_PREC_FP8_SPLIT = 4
GOAT_PREC_BF16_SPLIT8 = 5
GOAT_DIR_LOT = 0  # GOAT (Alg. 3): entropic OT direction
GOAT_DIR_LAP = 1  # FAQ (Alg. 1): exact linear-assignment direction
GOAT_TRACE_MAX = 256
GOAT_MLP_PARAMS = 641

EXPORTED = ["goat_default_params", "goat_strerror", "goat_workspace_bytes", "goat_workspace_bytes_host",
            "goat_workspace_bytes_ex", "goat_match", "goat_match_host",
            "goat_gradient", "goat_gradient_ex", "goat_sinkhorn", "goat_line_search", "goat_fw_update", "goat_project",
            "goat_objective", "goat_gemm_bf16_xyT", "goat_sinkhorn_noalloc", "goat_match_batched",
            "goat_workspace_bytes_batched", "goat_dual_features", "goat_mlp_forward", "goat_mlp_train_step",
            "goat_mlp_warm_start", "goat_lap_default_options", "goat_project_ex", "goat_entropic_eps",
            "goat_dual_targets"]


class GoatError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class goat_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("sk_max_iter", ctypes.c_int), ("sk_tol", ctypes.c_float),
                ("sk_warm_start", ctypes.c_int), ("sk_check_every", ctypes.c_int),
                ("project_on_grad", ctypes.c_int), ("lap_max_rounds", ctypes.c_int), ("profile", ctypes.c_int),
                ("mlp_weights", ctypes.c_void_p), ("direction", ctypes.c_int), ("maximize", ctypes.c_int),
                ("seeds", ctypes.c_int), ("directed", ctypes.c_int), ("relaxed_out", ctypes.c_void_p)]


class goat_stats(ctypes.Structure):
    _fields_ = [("fw_iters", ctypes.c_int), ("converged", ctypes.c_int), ("sk_iters_total", ctypes.c_int),
                ("sk_iters", ctypes.c_int * GOAT_TRACE_MAX), ("sk_resid", ctypes.c_float * GOAT_TRACE_MAX),
                ("alpha", ctypes.c_double * GOAT_TRACE_MAX), ("objective", ctypes.c_double),
                ("disagreements", ctypes.c_double), ("lap_gap", ctypes.c_double), ("lap_rounds", ctypes.c_int),
                ("ms_total", ctypes.c_float), ("ms_fw", ctypes.c_float), ("ms_project", ctypes.c_float),
                ("ms_gemm", ctypes.c_float), ("gemm_launches", ctypes.c_int), ("ms_sinkhorn", ctypes.c_float),
                ("ms_step", ctypes.c_float), ("launches", ctypes.c_longlong),
                ("lap_tail_bids", ctypes.c_longlong), ("lap_sap_rows", ctypes.c_int),
                ("lap_sap_pops", ctypes.c_longlong), ("lap_ms_head", ctypes.c_float),
                ("lap_ms_tail", ctypes.c_float), ("lap_ms_sap", ctypes.c_float)]


class goat_lap_options(ctypes.Structure):
    _fields_ = [("max_rounds", ctypes.c_int), ("head_rounds", ctypes.c_int), ("tail_bids", ctypes.c_longlong),
                ("tail_stall", ctypes.c_longlong), ("sap_pops", ctypes.c_longlong), ("head_stall", ctypes.c_int),
                ("sap_every_phase", ctypes.c_int)]


class goat_lap_info(ctypes.Structure):
    _fields_ = [("phases", ctypes.c_int), ("rounds", ctypes.c_int), ("tail_bids", ctypes.c_longlong),
                ("sap_rows", ctypes.c_int), ("sap_pops", ctypes.c_longlong), ("sap_steps", ctypes.c_longlong),
                ("filled", ctypes.c_int),
                ("ms_head", ctypes.c_double), ("ms_tail", ctypes.c_double), ("ms_sap", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_d = ctypes.c_double


def load():
    """Loads libgoat.so (built by ``paper_2111_05366_gb300._build``); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgoat.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_2111_05366_gb300._build` (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "goat_default_params": (None, [ctypes.POINTER(goat_params)]),
            "goat_strerror": (ctypes.c_char_p, [_i]),
            "goat_workspace_bytes": (ctypes.c_size_t, [_i, _i, _i]),
            "goat_workspace_bytes_host": (ctypes.c_size_t, [_i, _i, _i]),
            "goat_workspace_bytes_ex": (ctypes.c_size_t, [_i, _i, _i, _i, _i, _i]),
            "goat_match": (_i, [_vp, _vp, _i, _i, _vp, _f, _i, _f, ctypes.POINTER(goat_params), _vp,
                                ctypes.POINTER(_d), ctypes.POINTER(goat_stats), _vp, ctypes.c_size_t, _vp]),
            "goat_match_host": (_i, [_vp, _vp, _i, _i, _vp, _f, _i, _f, ctypes.POINTER(goat_params), _vp,
                                     ctypes.POINTER(_d), ctypes.POINTER(goat_stats), _vp, ctypes.c_size_t, _vp]),
            "goat_gradient": (_i, [_vp, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.c_size_t, _vp]),
            "goat_gradient_ex": (_i, [_vp, _vp, _i, _i, _vp, _vp, _i, _i, _vp, ctypes.c_size_t, _vp]),
            "goat_sinkhorn": (_i, [_vp, _i, _f, _f, _i, _vp, _vp, _vp, ctypes.POINTER(_i), ctypes.POINTER(_f), _vp,
                                   ctypes.c_size_t, _vp]),
            "goat_line_search": (_i, [_vp, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                      ctypes.POINTER(_d), _vp, ctypes.c_size_t, _vp]),
            "goat_fw_update": (_i, [_vp, _vp, _vp, _vp, _i, _d, _vp]),
            "goat_entropic_eps": (_i, [_vp, _i, _f, ctypes.POINTER(_f), _vp]),
            "goat_dual_targets": (_i, [_vp, _vp, _i, _f, _vp, _vp]),
            "goat_project": (_i, [_vp, _i, _i, _vp, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp, ctypes.c_size_t,
                                  _vp]),
            "goat_lap_default_options": (None, [ctypes.POINTER(goat_lap_options)]),
            "goat_project_ex": (_i, [_vp, _i, _i, ctypes.POINTER(goat_lap_options), _vp, ctypes.POINTER(_d),
                                     ctypes.POINTER(_d), ctypes.POINTER(goat_lap_info), _vp, ctypes.c_size_t, _vp]),
            "goat_objective": (_i, [_vp, _vp, _i, _i, _vp, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp,
                                    ctypes.c_size_t, _vp]),
            "goat_gemm_bf16_xyT": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _i, _f, _vp, _i, _i, _i, _vp]),
            "goat_sinkhorn_noalloc": (_i, [_vp, _i, _f, _f, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
            "goat_workspace_bytes_batched": (ctypes.c_size_t, [_vp, _i, _i]),
            "goat_dual_features": (_i, [_vp, _vp, _vp, _i, _i, _f, _vp, _vp, ctypes.c_size_t, _vp]),
            "goat_mlp_forward": (_i, [_vp, _vp, _i, _vp, _vp]),
            "goat_mlp_train_step": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _f, _i, _vp, _vp, _vp]),
            "goat_mlp_warm_start": (_i, [_vp, _vp, _vp, _i, _i, _f, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
            "goat_match_batched": (_i, [_vp, _vp, _vp, _vp, _i, _i, ctypes.c_ulonglong, _f, _i, _f,
                                        ctypes.POINTER(goat_params), _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                        _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(status: int) -> str:
    return load().goat_strerror(int(status)).decode()


def _check(status: int, where: str, allow=(GOAT_OK,)):
    if status not in allow:
        raise GoatError(status, where)
    return status


# ---------------------------------------------------------------- marshalling

def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype=None, shape=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _adj_dtype(A):
    torch = _torch()
    if A.dtype == torch.uint8:
        return GOAT_DTYPE_U8
    if A.dtype == torch.float32:
        return GOAT_DTYPE_F32
    raise TypeError("adjacency matrices must be uint8 (0/1) or float32")


def default_params(**overrides) -> goat_params:
    p = goat_params()
    load().goat_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        if k == "mlp_weights" and v is not None and not isinstance(v, int):
            v = _dev(v, _torch().bfloat16, (GOAT_MLP_PARAMS,), "mlp_weights").value
        if k == "relaxed_out" and v is not None and not isinstance(v, int):
            v = _dev(v, _torch().float32, None, "relaxed_out").value
        setattr(p, k, v)
    return p


def workspace_bytes(n: int, dtype_AB: int = GOAT_DTYPE_U8, precision: int = GOAT_PREC_BF16,
                    host: bool = False, directed: int = 0, seeds: int = 0) -> int:
    """Scratch bytes goat_match (host=False) or goat_match_host (host=True) needs for size n."""
    return int(load().goat_workspace_bytes_ex(int(n), int(dtype_AB), int(precision), int(directed), int(seeds),
                                              int(bool(host))))


def _stats_dict(st: goat_stats) -> dict:
    k = min(st.fw_iters, GOAT_TRACE_MAX)
    return {"fw_iters": st.fw_iters, "converged": bool(st.converged), "sk_iters_total": st.sk_iters_total,
            "sk_iters": list(st.sk_iters[:k]), "sk_resid": list(st.sk_resid[:k]), "alpha": list(st.alpha[:k]),
            "objective": st.objective, "disagreements": st.disagreements, "lap_gap": st.lap_gap,
            "lap_rounds": st.lap_rounds, "ms_total": st.ms_total, "ms_fw": st.ms_fw, "ms_project": st.ms_project,
            "ms_gemm": st.ms_gemm, "gemm_launches": st.gemm_launches, "ms_sinkhorn": st.ms_sinkhorn,
            "ms_step": st.ms_step, "launches": st.launches, "lap_tail_bids": st.lap_tail_bids,
            "lap_sap_rows": st.lap_sap_rows, "lap_sap_pops": st.lap_sap_pops, "lap_ms_head": st.lap_ms_head,
            "lap_ms_tail": st.lap_ms_tail, "lap_ms_sap": st.lap_ms_sap}


# ---------------------------------------------------------------- entry points

def goat_match(A, B, init=None, eps_rel: float = 0.03, max_iter: int = 30, tol: float = 0.03,
               params: goat_params | None = None, workspace=None):
    """Whole GOAT solve (Alg. 3) on device tensors A, B (n x n, uint8 or float32), or
    FAQ (Alg. 1) with params.direction = GOAT_DIR_LAP.

    Returns (perm int32 numpy [n], objective, stats dict)."""
    n = A.shape[0]
    dt = _adj_dtype(A)
    a = _dev(A, A.dtype, (n, n), "A")
    b = _dev(B, A.dtype, (n, n), "B")
    ini = _dev(init, _torch().float32, (n, n), "init") if init is not None else None
    perm = np.empty(n, dtype=np.int32)
    obj = ctypes.c_double()
    st = goat_stats()
    p = params if params is not None else default_params()
    ws = _dev(workspace, None, None, "workspace") if workspace is not None else None
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    r = load().goat_match(a, b, n, dt, ini, float(eps_rel), int(max_iter), float(tol), ctypes.byref(p),
                          perm.ctypes.data_as(ctypes.c_void_p), ctypes.byref(obj), ctypes.byref(st), ws, wsb,
                          _stream())
    _check(r, "goat_match")
    return perm, obj.value, _stats_dict(st)


def goat_match_host(A, B, init=None, eps_rel: float = 0.03, max_iter: int = 30, tol: float = 0.03,
                    params: goat_params | None = None, workspace=None):
    """GOAT solve from HOST numpy arrays (the copies to the device are part of the call)."""
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    if A.dtype == np.uint8:
        dt = GOAT_DTYPE_U8
    elif A.dtype == np.float32:
        dt = GOAT_DTYPE_F32
    else:
        raise TypeError("A must be uint8 or float32")
    if B.dtype != A.dtype or A.shape != B.shape or A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A and B must be square arrays of the same shape and dtype")
    n = A.shape[0]
    ini = np.ascontiguousarray(init, dtype=np.float32) if init is not None else None
    perm = np.empty(n, dtype=np.int32)
    obj = ctypes.c_double()
    st = goat_stats()
    p = params if params is not None else default_params()
    ws = _dev(workspace, None, None, "workspace") if workspace is not None else None
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    r = load().goat_match_host(A.ctypes.data_as(ctypes.c_void_p), B.ctypes.data_as(ctypes.c_void_p), n, dt,
                               ini.ctypes.data_as(ctypes.c_void_p) if ini is not None else None, float(eps_rel),
                               int(max_iter), float(tol), ctypes.byref(p), perm.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(obj), ctypes.byref(st), ws, wsb, _stream())
    _check(r, "goat_match_host")
    return perm, obj.value, _stats_dict(st)


def goat_gradient(A, B, P, precision: int = GOAT_PREC_BF16, out=None, directed: bool = False):
    """G = -grad f(P) (Alg. 3 step 1) on the tensor cores: -2 A P B for symmetric graphs,
    -(A P B^T + A^T P B) with directed=True.  Returns a float32 tensor."""
    torch = _torch()
    n = A.shape[0]
    G = out if out is not None else torch.empty((n, n), dtype=torch.float32, device=A.device)
    r = load().goat_gradient_ex(_dev(A, A.dtype, (n, n), "A"), _dev(B, A.dtype, (n, n), "B"), n, _adj_dtype(A),
                                _dev(P, torch.float32, (n, n), "P"), _dev(G, torch.float32, (n, n), "G"),
                                int(precision), int(bool(directed)), None, 0, _stream())
    _check(r, "goat_gradient")
    return G


def goat_sinkhorn(G, eps: float, tol: float, max_iter: int, g_init=None, want_Q: bool = False):
    """LOT (Alg. 2): log-domain Sinkhorn on exp(-G/eps).  Returns (f, g, Q or None, iters, resid)."""
    torch = _torch()
    n = G.shape[0]
    f = torch.empty(n, dtype=torch.float32, device=G.device)
    g = (g_init.clone() if g_init is not None else torch.zeros(n, dtype=torch.float32, device=G.device))
    Q = torch.empty((n, n), dtype=torch.float32, device=G.device) if want_Q else None
    it = ctypes.c_int()
    res = ctypes.c_float()
    r = load().goat_sinkhorn(_dev(G, torch.float32, (n, n), "G"), n, float(eps), float(tol), int(max_iter),
                             _dev(f, torch.float32, (n,), "f"), _dev(g, torch.float32, (n,), "g"),
                             _dev(Q, torch.float32, (n, n), "Q") if Q is not None else None, ctypes.byref(it),
                             ctypes.byref(res), None, 0, _stream())
    _check(r, "goat_sinkhorn")
    return f, g, Q, it.value, res.value


def goat_line_search(G, G_Q, P, Q, maximize: bool = True):
    """Exact quadratic step (Alg. 3 step 3).  Returns (alpha, a, b); alpha weights Q."""
    torch = _torch()
    n = G.shape[0]
    al, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    sh = (n, n)
    r = load().goat_line_search(_dev(G, torch.float32, sh, "G"), _dev(G_Q, torch.float32, sh, "G_Q"),
                                _dev(P, torch.float32, sh, "P"), _dev(Q, torch.float32, sh, "Q"), n,
                                int(bool(maximize)), ctypes.byref(al), ctypes.byref(a), ctypes.byref(b), None, 0,
                                _stream())
    _check(r, "goat_line_search")
    return al.value, a.value, b.value


def goat_fw_update(P, G, Q, G_Q, alpha: float):
    """In place: P += alpha (Q - P), G += alpha (G_Q - G) (Alg. 3 step 4)."""
    torch = _torch()
    n = P.shape[0]
    sh = (n, n)
    r = load().goat_fw_update(_dev(P, torch.float32, sh, "P"), _dev(G, torch.float32, sh, "G"),
                              _dev(Q, torch.float32, sh, "Q"), _dev(G_Q, torch.float32, sh, "G_Q"), n, float(alpha),
                              _stream())
    _check(r, "goat_fw_update")


def goat_entropic_eps(G, eps_rel: float = 0.03) -> float:
    """The entropic weight goat_match uses for cost G: eps_rel * max|G| (1 if G == 0)."""
    torch = _torch()
    n = G.shape[0]
    e = _f()
    r = load().goat_entropic_eps(_dev(G, torch.float32, (n, n), "G"), n, float(eps_rel), ctypes.byref(e), _stream())
    _check(r, "goat_entropic_eps")
    return e.value


def goat_dual_targets(f, g, eps: float):
    """Training targets [f/eps - mean, g/eps - mean] (2n floats) of converged duals."""
    torch = _torch()
    n = f.shape[0]
    t = torch.empty(2 * n, dtype=torch.float32, device=f.device)
    r = load().goat_dual_targets(_dev(f, torch.float32, (n,), "f"), _dev(g, torch.float32, (n,), "g"), n,
                                 float(eps), _dev(t, torch.float32, (2 * n,), "t"), _stream())
    _check(r, "goat_dual_targets")
    return t


def goat_project(M, maximize: bool = True, allow_uncertified: bool = False):
    """Linear assignment on the GPU (auction + LP-duality certification).

    Returns (perm int32 tensor, cost, gap) with cost = sum_i M[i, perm i] in FP64."""
    torch = _torch()
    n = M.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device=M.device)
    cost, gap = ctypes.c_double(), ctypes.c_double()
    r = load().goat_project(_dev(M, torch.float32, (n, n), "M"), n, int(bool(maximize)),
                            _dev(perm, torch.int32, (n,), "perm"), ctypes.byref(cost), ctypes.byref(gap), None, 0,
                            _stream())
    allow = (GOAT_OK, GOAT_ERR_NOT_CONVERGED) if allow_uncertified else (GOAT_OK,)
    _check(r, "goat_project", allow)
    return perm, cost.value, gap.value


def lap_options(**overrides) -> goat_lap_options:
    """The projection's default schedule with `overrides` applied (see goat_lap_options)."""
    o = goat_lap_options()
    load().goat_lap_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def goat_project_ex(M, maximize: bool = True, options=None, allow_uncertified: bool = False):
    """goat_project with an explicit schedule; returns (perm, cost, gap, info dict)."""
    torch = _torch()
    n = M.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device=M.device)
    cost, gap = ctypes.c_double(), ctypes.c_double()
    info = goat_lap_info()
    opt = ctypes.byref(options) if options is not None else None
    r = load().goat_project_ex(_dev(M, torch.float32, (n, n), "M"), n, int(bool(maximize)), opt,
                               _dev(perm, torch.int32, (n,), "perm"), ctypes.byref(cost), ctypes.byref(gap),
                               ctypes.byref(info), None, 0, _stream())
    allow = (GOAT_OK, GOAT_ERR_NOT_CONVERGED) if allow_uncertified else (GOAT_OK,)
    _check(r, "goat_project_ex", allow)
    return perm, cost.value, gap.value, {f: getattr(info, f) for f, _ in goat_lap_info._fields_}


def goat_objective(A, B, perm):
    """f(perm) = sum_ij A_ij B[perm i, perm j] and the disagreement count (exact for uint8)."""
    torch = _torch()
    n = A.shape[0]
    obj, dis = ctypes.c_double(), ctypes.c_double()
    r = load().goat_objective(_dev(A, A.dtype, (n, n), "A"), _dev(B, A.dtype, (n, n), "B"), n, _adj_dtype(A),
                              _dev(perm, torch.int32, (n,), "perm"), ctypes.byref(obj), ctypes.byref(dis), None, 0,
                              _stream())
    _check(r, "goat_objective")
    return obj.value, dis.value


def goat_gemm_bf16_xyT(X, Y, k_total: int, kx_period: int, scale: float = 1.0, out_rows=None, out_cols=None):
    """out = scale * X[:, k mod kx_period] Y[:, k]^T on the tensor cores (kernel-level entry)."""
    torch = _torch()
    xr, xs = X.shape
    yr, ys = Y.shape
    orows = xr if out_rows is None else out_rows
    ocols = yr if out_cols is None else out_cols
    out = torch.empty((orows, ocols), dtype=torch.float32, device=X.device)
    r = load().goat_gemm_bf16_xyT(_dev(X, torch.bfloat16, None, "X"), xr, xs, int(kx_period),
                                  _dev(Y, torch.bfloat16, None, "Y"), yr, ys, int(k_total), float(scale),
                                  _dev(out, torch.float32, None, "out"), ocols, orows, ocols, _stream())
    _check(r, "goat_gemm_bf16_xyT")
    return out


NOALLOC_MAX_N = 4096
NOALLOC_MAX_ITER = 1000


def goat_sinkhorn_noalloc(G, eps: float, tol: float, max_iter: int, g_init=None):
    """goat_sinkhorn for callers that cannot allocate device memory during the call.

    The library side allocates nothing and does not synchronise with the device;
    this wrapper creates the output tensors itself for convenience (a caller that
    cannot allocate passes preallocated f, g, iters, resid, status through the C
    ABI).  n <= NOALLOC_MAX_N, max_iter <= NOALLOC_MAX_ITER.  Returns
    (f, g, iters, resid, status) with iters / resid / status as one-element
    device tensors (status: GOAT_OK or GOAT_ERR_NAN)."""
    torch = _torch()
    n = G.shape[0]
    if n > NOALLOC_MAX_N:
        raise ValueError(f"n = {n} exceeds the no-allocation maximum of {NOALLOC_MAX_N}")
    if max_iter > NOALLOC_MAX_ITER:
        raise ValueError(f"max_iter = {max_iter} exceeds the no-allocation maximum of {NOALLOC_MAX_ITER}")
    f = torch.empty(n, dtype=torch.float32, device=G.device)
    g = (g_init.clone() if g_init is not None else torch.zeros(n, dtype=torch.float32, device=G.device))
    it = torch.zeros(1, dtype=torch.int32, device=G.device)
    res = torch.zeros(1, dtype=torch.float32, device=G.device)
    status = torch.zeros(1, dtype=torch.int32, device=G.device)
    r = load().goat_sinkhorn_noalloc(_dev(G, torch.float32, (n, n), "G"), n, float(eps), float(tol), int(max_iter),
                                     _dev(f, torch.float32, (n,), "f"), _dev(g, torch.float32, (n,), "g"),
                                     _dev(it, torch.int32, (1,), "iters"), _dev(res, torch.float32, (1,), "resid"),
                                     _dev(status, torch.int32, (1,), "status"), _stream())
    _check(r, "goat_sinkhorn_noalloc")
    return f, g, it, res, status


BATCH_MAX_N = 2048


def goat_match_batched(As, Bs, restarts: int = 1, seed: int = 0, eps_rel: float = 0.03, max_iter: int = 30,
                       tol: float = 0.03, params: goat_params | None = None, device_AB=None, want_relaxed=False):
    """Batched GOAT: lists of uint8 numpy matrices (pairs of uneven n), `restarts` starts each.

    The pairs are packed into one device buffer here (marshalling); all arithmetic
    runs in libgoat.  `device_AB` may pass an already packed (A, B, adj_off, n)
    tuple of device tensors / host arrays to keep the copy out of a timed region.
    Returns (list of perms, objectives, best restarts, FW iterations), plus the list of
    every problem's final relaxed P (problem order pair * restarts + restart) when
    want_relaxed is set."""
    torch = _torch()
    if device_AB is None:
        ns = np.array([a.shape[0] for a in As], dtype=np.int32)
        off = np.zeros(len(As), dtype=np.int64)
        off[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
        Ah = np.concatenate([np.ascontiguousarray(a, dtype=np.uint8).ravel() for a in As])
        Bh = np.concatenate([np.ascontiguousarray(b_, dtype=np.uint8).ravel() for b_ in Bs])
        Ad = torch.from_numpy(Ah).cuda()
        Bd = torch.from_numpy(Bh).cuda()
    else:
        Ad, Bd, off, ns = device_AB
    num = len(ns)
    perm = np.empty(int(ns.sum()), dtype=np.int32)
    obj = np.empty(num, dtype=np.float64)
    best = np.empty(num, dtype=np.int32)
    its = np.empty(num, dtype=np.int32)
    p = params if params is not None else default_params()
    rel = None
    if want_relaxed:
        rel = torch.empty(int((ns.astype(np.int64) ** 2).sum()) * restarts, dtype=torch.float32, device=Ad.device)
    r = load().goat_match_batched(_dev(Ad, torch.uint8, None, "A"), _dev(Bd, torch.uint8, None, "B"),
                                  off.ctypes.data_as(ctypes.c_void_p), ns.ctypes.data_as(ctypes.c_void_p), num,
                                  int(restarts), ctypes.c_ulonglong(seed), float(eps_rel), int(max_iter),
                                  float(tol), ctypes.byref(p), perm.ctypes.data_as(ctypes.c_void_p),
                                  obj.ctypes.data_as(ctypes.c_void_p), best.ctypes.data_as(ctypes.c_void_p),
                                  its.ctypes.data_as(ctypes.c_void_p),
                                  _dev(rel, torch.float32, None, "relaxed") if rel is not None else None, None, 0,
                                  _stream())
    _check(r, "goat_match_batched")
    cuts = np.cumsum(ns)[:-1]
    out = (np.split(perm, cuts), obj, best, its)
    if want_relaxed:
        mats, o = [], 0
        relh = rel.cpu().numpy()
        for k in range(num):
            for _ in range(restarts):
                m = int(ns[k]) ** 2
                mats.append(relh[o:o + m].reshape(int(ns[k]), int(ns[k])))
                o += m
        out = out + (mats,)
    return out


# ---------------------------------------------------------------- learned warm start

def goat_dual_features(G, A, B, eps: float):
    """Per-node features (2n x 8 float32 tensor) of the learned Sinkhorn warm start."""
    torch = _torch()
    n = G.shape[0]
    F = torch.empty((2 * n, 8), dtype=torch.float32, device=G.device)
    r = load().goat_dual_features(_dev(G, torch.float32, (n, n), "G"), _dev(A, A.dtype, (n, n), "A"),
                                  _dev(B, A.dtype, (n, n), "B"), n, _adj_dtype(A), float(eps),
                                  _dev(F, torch.float32, (2 * n, 8), "feats"), None, 0, _stream())
    _check(r, "goat_dual_features")
    return F


def goat_mlp_forward(weights_bf16, x):
    """Network outputs for feature rows x (N x 8): predicted duals over eps."""
    torch = _torch()
    N = x.shape[0]
    y = torch.empty(N, dtype=torch.float32, device=x.device)
    r = load().goat_mlp_forward(_dev(weights_bf16, torch.bfloat16, (GOAT_MLP_PARAMS,), "weights"),
                                _dev(x, torch.float32, (N, 8), "x"), N, _dev(y, torch.float32, (N,), "y"), _stream())
    _check(r, "goat_mlp_forward")
    return y


def goat_mlp_train_step(master, adam_state, weights_bf16, x, t, lr: float, step: int, grad=None, loss=None):
    """One training step (loss, gradient at the BF16 weights, Adam update when lr > 0)."""
    torch = _torch()
    N = x.shape[0]
    grad = grad if grad is not None else torch.empty(GOAT_MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=x.device)
    r = load().goat_mlp_train_step(_dev(master, torch.float32, (GOAT_MLP_PARAMS,), "master"),
                                   _dev(adam_state, torch.float32, (2 * GOAT_MLP_PARAMS,), "adam_state"),
                                   _dev(weights_bf16, torch.bfloat16, (GOAT_MLP_PARAMS,), "weights"),
                                   _dev(x, torch.float32, (N, 8), "x"), _dev(t, torch.float32, (N,), "t"), N,
                                   float(lr), int(step), _dev(loss, torch.float32, (1,), "loss"),
                                   _dev(grad, torch.float32, (GOAT_MLP_PARAMS,), "grad"), _stream())
    _check(r, "goat_mlp_train_step")
    return loss, grad


def goat_mlp_warm_start(G, A, B, eps: float, weights_bf16):
    """Warm-start column duals g (n, float32) predicted by the network for goat_sinkhorn."""
    torch = _torch()
    n = G.shape[0]
    g = torch.empty(n, dtype=torch.float32, device=G.device)
    r = load().goat_mlp_warm_start(_dev(G, torch.float32, (n, n), "G"), _dev(A, A.dtype, (n, n), "A"),
                                   _dev(B, A.dtype, (n, n), "B"), n, _adj_dtype(A), float(eps),
                                   _dev(weights_bf16, torch.bfloat16, (GOAT_MLP_PARAMS,), "weights"),
                                   _dev(g, torch.float32, (n,), "g"), None, 0, _stream())
    _check(r, "goat_mlp_warm_start")
    return g

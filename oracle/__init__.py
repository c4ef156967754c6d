"""FP64 CPU oracle for GOAT / FAQ -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference arms may import this package.  The GPU library never uses it and
it never uses the GPU library: the two share no code.

The arithmetic lives in ``goat_oracle.c`` (plain C, FP64, naive loops); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Each wrapper names the part of the paper it follows (Alg. 1-3,
eq. QAP, Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "goat_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgoat_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class OracleStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("objective", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile goat_oracle.c into libgoat_oracle.so next to it (gcc, -O2, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "oracle_objective": (ctypes.c_double, [_dp, _dp, _dp, ctypes.c_int]),
            "oracle_objective_perm": (ctypes.c_double, [_dp, _dp, ctypes.c_int, _ip]),
            "oracle_objective_perm_u8": (ctypes.c_int64, [_u8p, _u8p, ctypes.c_int, _ip]),
            "oracle_gradient": (None, [_dp, _dp, _dp, ctypes.c_int, _dp]),
            "oracle_gradient_rows_u8": (None, [_u8p, _u8p, _fp, ctypes.c_int, _ip, ctypes.c_int, _dp]),
            "oracle_gradient_rows_f32": (None, [_fp, _fp, _fp, ctypes.c_int, _ip, ctypes.c_int, _dp]),
            "oracle_sinkhorn_knopp": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                                     _dp, _dp, _dp, _dp]),
            "oracle_lot": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          _dp, _dp, _dp, _dp, _dp]),
            "oracle_lot_log": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, _dp, _dp, _dp, _dp]),
            "oracle_lot_rows_f32": (None, [_fp, ctypes.c_int, ctypes.c_int, _fp, ctypes.c_double, _dp]),
            "oracle_lot_colsums_f32": (None, [_fp, ctypes.c_int, ctypes.c_int, _fp, _fp, ctypes.c_double, _dp]),
            "oracle_step_size": (ctypes.c_double, [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]),
            "oracle_lap_min": (ctypes.c_double, [_dp, ctypes.c_int, _ip, _dp, _dp]),
            "oracle_lap": (ctypes.c_double, [_dp, ctypes.c_int, ctypes.c_int, _ip]),
            "oracle_lap_f32": (ctypes.c_double, [_fp, ctypes.c_int, ctypes.c_int, _ip]),
            "oracle_assignment_cost_f32": (ctypes.c_double, [_fp, ctypes.c_int, _ip]),
            "oracle_lap_certificate_f32": (None, [_fp, ctypes.c_int, _ip, _dp, _dp, _dp, _dp]),
            "oracle_brute_lap": (ctypes.c_double, [_dp, ctypes.c_int, ctypes.c_int, _ip, _ip]),
            "oracle_random_start": (None, [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _dp]),
            "oracle_splitmix64_output": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
            "oracle_dual_features": (None, [_dp, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp]),
            "oracle_mlp_loss_grad": (ctypes.c_double, [_dp, _dp, _dp, ctypes.c_int, _dp, _dp]),
            "oracle_brute_qap": (ctypes.c_double, [_dp, _dp, ctypes.c_int, ctypes.c_int, _ip]),
            "oracle_goat": (ctypes.c_int, [_dp, _dp, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _ip,
                                           ctypes.POINTER(OracleStats)]),
            "oracle_goat_seeded": (ctypes.c_int, [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _ip,
                                                  ctypes.POINTER(OracleStats)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ---------------------------------------------------------------- marshalling

def _d(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _f(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float32)


def _i(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.int32)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _square(*mats) -> int:
    n = mats[0].shape[0]
    for m in mats:
        if m.shape != (n, n):
            raise ValueError(f"expected {n}x{n} matrices, got {m.shape}")
    return n


# ---------------------------------------------------------------- wrappers

def objective(A, B, P) -> float:
    """f(P) = tr(A^T P B P^T), eq. (QAP)."""
    A, B, P = _d(A), _d(B), _d(P)
    n = _square(A, B, P)
    return _load().oracle_objective(_ptr(A, _dp), _ptr(B, _dp), _ptr(P, _dp), n)


def objective_perm(A, B, perm) -> float:
    """f at the permutation matrix with P[i, perm[i]] = 1: sum_ij A_ij B[perm i, perm j]."""
    A, B, perm = _d(A), _d(B), _i(perm)
    n = _square(A, B)
    return _load().oracle_objective_perm(_ptr(A, _dp), _ptr(B, _dp), n, _ptr(perm, _ip))


def objective_perm_u8(A, B, perm) -> int:
    """Exact integer f(perm) on byte adjacency matrices."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    perm = _i(perm)
    n = _square(A, B)
    return int(_load().oracle_objective_perm_u8(_ptr(A, _u8p), _ptr(B, _u8p), n, _ptr(perm, _ip)))


def gradient(A, B, P) -> np.ndarray:
    """grad f(P) = A P B^T + A^T P B (Alg. 1 / Alg. 3, step 1), naive loops."""
    A, B, P = _d(A), _d(B), _d(P)
    n = _square(A, B, P)
    out = np.empty((n, n), dtype=np.float64)
    _load().oracle_gradient(_ptr(A, _dp), _ptr(B, _dp), _ptr(P, _dp), n, _ptr(out, _dp))
    return out


def gradient_rows(A, B, P, rows) -> np.ndarray:
    """Selected rows of grad f(P) for large n (byte or float adjacency, float32 P)."""
    rows = _i(rows)
    P = _f(P)
    n = P.shape[0]
    out = np.empty((len(rows), n), dtype=np.float64)
    if np.asarray(A).dtype == np.uint8 and np.asarray(B).dtype == np.uint8:
        A = np.ascontiguousarray(A)
        B = np.ascontiguousarray(B)
        _load().oracle_gradient_rows_u8(_ptr(A, _u8p), _ptr(B, _u8p), _ptr(P, _fp), n, _ptr(rows, _ip),
                                        len(rows), _ptr(out, _dp))
    else:
        A, B = _f(A), _f(B)
        _load().oracle_gradient_rows_f32(_ptr(A, _fp), _ptr(B, _fp), _ptr(P, _fp), n, _ptr(rows, _ip),
                                         len(rows), _ptr(out, _dp))
    return out


def sinkhorn_knopp(K, tol: float, max_iter: int, v_init=None):
    """Sinkhorn-Knopp scaling of a positive kernel K to marginals 1_n.

    Returns (Q, u, v, iters, resid)."""
    K = _d(K)
    n = _square(K)
    Q = np.empty((n, n)); u = np.empty(n); v = np.empty(n)
    r = ctypes.c_double()
    vi = _d(v_init) if v_init is not None else None
    it = _load().oracle_sinkhorn_knopp(_ptr(K, _dp), n, tol, max_iter,
                                       _ptr(vi, _dp) if vi is not None else None,
                                       _ptr(Q, _dp), _ptr(u, _dp), _ptr(v, _dp), ctypes.byref(r))
    return Q, u, v, it, r.value


def lot(M, eps: float, tol: float, max_iter: int, g_init=None):
    """LOT (Alg. 2): min <Q, M> - eps H(Q) over doubly stochastic Q, scaling domain.

    Returns (Q, f, g, iters, resid) with Q_ij = exp((f_i + g_j - M_ij) / eps)."""
    M = _d(M)
    n = _square(M)
    Q = np.empty((n, n)); f = np.empty(n); g = np.empty(n)
    r = ctypes.c_double()
    gi = _d(g_init) if g_init is not None else None
    it = _load().oracle_lot(_ptr(M, _dp), n, eps, tol, max_iter, _ptr(gi, _dp) if gi is not None else None,
                            _ptr(Q, _dp), _ptr(f, _dp), _ptr(g, _dp), ctypes.byref(r))
    return Q, f, g, it, r.value


def lot_log(M, eps: float, tol: float, max_iter: int, g_init=None):
    """LOT in the log domain; g_init warm-starts the column duals (default 0)."""
    M = _d(M)
    n = _square(M)
    f = np.zeros(n)
    g = _d(g_init).copy() if g_init is not None else np.zeros(n)
    Q = np.empty((n, n))
    r = ctypes.c_double()
    it = _load().oracle_lot_log(_ptr(M, _dp), n, eps, tol, max_iter, _ptr(f, _dp), _ptr(g, _dp),
                                _ptr(Q, _dp), ctypes.byref(r))
    return Q, f, g, it, r.value


def lot_rows(M_rows, g, eps: float) -> np.ndarray:
    """Row scaling f_r = -eps LSE_j((g_j - M_rj)/eps) on a block of rows (nrows x n), FP64."""
    M_rows, g = _f(M_rows), _f(g)
    nrows, n = M_rows.shape
    out = np.empty(nrows)
    _load().oracle_lot_rows_f32(_ptr(M_rows, _fp), nrows, n, _ptr(g, _fp), eps, _ptr(out, _dp))
    return out


def lot_colsums(M_cols, f, g_cols, eps: float) -> np.ndarray:
    """Column sums sum_i exp((f_i + g_c - M_ic)/eps) on a block of columns (n x ncols), FP64."""
    M_cols, f, g_cols = _f(M_cols), _f(f), _f(g_cols)
    n, ncols = M_cols.shape
    out = np.empty(ncols)
    _load().oracle_lot_colsums_f32(_ptr(M_cols, _fp), n, ncols, _ptr(f, _fp), _ptr(g_cols, _fp), eps,
                                   _ptr(out, _dp))
    return out


def step_size(A, B, P, Q, maximize: bool = True):
    """Alg. 3 step 3: alpha in argmax_{[0,1]} f(alpha P + (1-alpha) Q) (paper's notation).

    Returns (alpha, a, b) where f(alpha P + (1-alpha) Q) = f(Q) + b alpha + a alpha^2."""
    A, B, P, Q = _d(A), _d(B), _d(P), _d(Q)
    n = _square(A, B, P, Q)
    a = ctypes.c_double(); b = ctypes.c_double()
    alpha = _load().oracle_step_size(_ptr(A, _dp), _ptr(B, _dp), _ptr(P, _dp), _ptr(Q, _dp), n,
                                     int(bool(maximize)), ctypes.byref(a), ctypes.byref(b))
    return alpha, a.value, b.value


def lap(C, maximize: bool = True):
    """Hungarian method (shortest augmenting paths with potentials).  Returns (perm, cost)."""
    C = np.asarray(C)
    n = _square(C)
    perm = np.empty(n, dtype=np.int32)
    if C.dtype == np.float32:
        C = np.ascontiguousarray(C)
        cost = _load().oracle_lap_f32(_ptr(C, _fp), n, int(bool(maximize)), _ptr(perm, _ip))
    else:
        C = _d(C)
        cost = _load().oracle_lap(_ptr(C, _dp), n, int(bool(maximize)), _ptr(perm, _ip))
    return perm, cost


def lap_min_with_duals(C):
    """Min-cost LAP returning (perm, cost, u, v) with reduced costs C - u - v >= 0."""
    C = _d(C)
    n = _square(C)
    perm = np.empty(n, dtype=np.int32); u = np.empty(n); v = np.empty(n)
    cost = _load().oracle_lap_min(_ptr(C, _dp), n, _ptr(perm, _ip), _ptr(u, _dp), _ptr(v, _dp))
    return perm, cost, u, v


def assignment_cost_f32(C, perm) -> float:
    """sum_i C[i, perm i] in FP64, row order, on a float32 matrix."""
    C, perm = _f(C), _i(perm)
    return _load().oracle_assignment_cost_f32(_ptr(C, _fp), C.shape[0], _ptr(perm, _ip))


def lap_certificate(C, perm, u, v):
    """(max_violation, gap) of duals (u, v) for the max-LAP on float32 C (see goat_oracle.c)."""
    C, perm, u, v = _f(C), _i(perm), _d(u), _d(v)
    mv = ctypes.c_double(); gap = ctypes.c_double()
    _load().oracle_lap_certificate_f32(_ptr(C, _fp), C.shape[0], _ptr(perm, _ip), _ptr(u, _dp), _ptr(v, _dp),
                                       ctypes.byref(mv), ctypes.byref(gap))
    return mv.value, gap.value


def splitmix64(seed: int, k: int) -> int:
    """Output number k of SplitMix64 seeded with `seed` (counter form)."""
    return int(_load().oracle_splitmix64_output(seed, k))


def random_start(n: int, seed: int, q: int) -> np.ndarray:
    """The paper's random start (J + K)/2 (Sec. 3.4), K = Sinkhorn-Knopp of SplitMix64 noise."""
    out = np.empty((n, n))
    _load().oracle_random_start(n, seed, q, _ptr(out, _dp))
    return out


def brute_lap(C, maximize: bool = True):
    """Exhaustive LAP over all n! permutations (n <= 10). Returns (cost, perm, n_optimal)."""
    C = _d(C)
    n = _square(C)
    if n > 10:
        raise ValueError("brute force is limited to n <= 10")
    perm = np.empty(n, dtype=np.int32)
    cnt = ctypes.c_int()
    cost = _load().oracle_brute_lap(_ptr(C, _dp), n, int(bool(maximize)), _ptr(perm, _ip), ctypes.byref(cnt))
    return cost, perm, cnt.value


def brute_qap(A, B, maximize: bool = True):
    """Exhaustive QAP / GM over all n! permutations (n <= 10). Returns (f*, perm)."""
    A, B = _d(A), _d(B)
    n = _square(A, B)
    if n > 10:
        raise ValueError("brute force is limited to n <= 10")
    perm = np.empty(n, dtype=np.int32)
    best = _load().oracle_brute_qap(_ptr(A, _dp), _ptr(B, _dp), n, int(bool(maximize)), _ptr(perm, _ip))
    return best, perm


def goat(A, B, P0=None, eps_rel: float = 0.03, max_iter: int = 30, tol: float = 0.03, sk_tol: float = 1e-3,
         sk_max_iter: int = 500, use_lap: bool = False, maximize: bool = True, project_on_grad: bool = False,
         seeds: int = 0):
    """GOAT (Alg. 3; use_lap=False) or FAQ (Alg. 1; use_lap=True) in FP64.

    seeds = m > 0: seeded graph matching (Fishkind et al., applied in Sec. 4): vertex
    i of A is known to match vertex i of B for i < m, and only the rest is solved.

    Returns a dict with perm, P (final relaxed iterate), alphas (paper's notation),
    sinkhorn_iters, iters, converged, objective."""
    A, B = _d(A), _d(B)
    n = _square(A, B)
    P0a = _d(P0) if P0 is not None else None
    perm = np.empty(n, dtype=np.int32)
    P = np.empty((n, n))
    alphas = np.zeros(max(max_iter, 1))
    sk = np.zeros(max(max_iter, 1), dtype=np.int32)
    st = OracleStats()
    if not 0 <= seeds <= n:
        raise ValueError(f"seeds must lie in [0, {n}]")
    _load().oracle_goat_seeded(_ptr(A, _dp), _ptr(B, _dp), n, int(seeds),
                               _ptr(P0a, _dp) if P0a is not None else None, eps_rel, max_iter, tol, sk_tol,
                               sk_max_iter, int(bool(use_lap)), int(bool(maximize)), int(bool(project_on_grad)),
                               _ptr(perm, _ip), _ptr(P, _dp), _ptr(alphas, _dp), _ptr(sk, _ip), ctypes.byref(st))
    return {"perm": perm, "P": P, "alphas": alphas[:st.iters], "sinkhorn_iters": sk[:st.iters],
            "iters": st.iters, "converged": bool(st.converged), "objective": st.objective}


def faq(A, B, **kw):
    """FAQ (Alg. 1): GOAT with the Hungarian LAP as the direction step."""
    return goat(A, B, use_lap=True, **kw)


def dual_features(G, A, B, eps: float) -> np.ndarray:
    """Per-node features of the learned warm start (2n x 8), from their definitions."""
    G, A, B = _d(G), _d(A), _d(B)
    n = _square(G, A, B)
    out = np.empty((2 * n, 8))
    _load().oracle_dual_features(_ptr(G, _dp), _ptr(A, _dp), _ptr(B, _dp), n, eps, _ptr(out, _dp))
    return out


def mlp_loss_grad(params, x, t):
    """(loss, gradient[641], outputs) of the warm-start network's mean squared error, FP64."""
    params, x, t = _d(params), _d(x), _d(t)
    N = x.shape[0]
    grad = np.empty(641)
    y = np.empty(N)
    L = _load().oracle_mlp_loss_grad(_ptr(params, _dp), _ptr(x, _dp), _ptr(t, _dp), N, _ptr(grad, _dp),
                                     _ptr(y, _dp))
    return L, grad, y

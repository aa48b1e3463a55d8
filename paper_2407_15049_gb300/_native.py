"""ctypes binding of liblorads.so (include/lorads.h), argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch
tensors and numpy arrays to pointers and sizes and turns status codes into
exceptions.  It raises at import of the library when ``liblorads.so`` has not
been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
LIB_PATH = Path(os.environ.get("LORADS_LIB", _HERE / "liblorads.so"))

LORADS_OK = 0
STATUS_NAMES = {
    0: "LORADS_OK", 1: "LORADS_ERR_INVALID_ARG", 2: "LORADS_ERR_NOT_SYMMETRIC", 3: "LORADS_ERR_OOM",
    4: "LORADS_ERR_CUDA", 5: "LORADS_ERR_NUMERIC", 6: "LORADS_ERR_MAXITER", 7: "LORADS_ERR_TIMEOUT",
    8: "LORADS_ERR_UNSUPPORTED",
}
LORADS_FP64, LORADS_FP32, LORADS_BF16, LORADS_MIXED, LORADS_DF64, LORADS_MIXED_BF16 = 0, 1, 2, 3, 4, 5


class LoradsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lorads_params(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("time_limit", C.c_double), ("lbfgs_mem", C.c_int32),
        ("max_inner", C.c_int32), ("max_outer", C.c_int32), ("rank_update_threshold", C.c_int32),
        ("rho0", C.c_double), ("rho_growth", C.c_double), ("rho_max", C.c_double),
        ("infeas_decrease", C.c_double), ("inner_rel", C.c_double), ("inner_progress", C.c_double),
        ("prec", C.c_int32),
        ("check_every", C.c_int32), ("seed", C.c_uint64), ("compute_err2", C.c_int32),
        ("lanczos_steps", C.c_int32), ("verbose", C.c_int32), ("reserved", C.c_int32),
        ("lbfgs_scaling", C.c_int32), ("rho_policy", C.c_int32), ("kernel_variant", C.c_int32),
        ("inner_scale", C.c_int32), ("admm_switch", C.c_double), ("cg_rel", C.c_double), ("cg_max", C.c_int32),
        ("admm_max_iter", C.c_int32), ("reopt_level", C.c_int32), ("max_reopt", C.c_int32),
        ("reopt_factor", C.c_double),
    ]


class lorads_result(C.Structure):
    _fields_ = [
        ("primal_obj", C.c_double), ("dual_obj", C.c_double), ("err1", C.c_double),
        ("err2", C.c_double), ("err3", C.c_double), ("sigma_min", C.c_double), ("rho", C.c_double),
        ("seconds", C.c_double), ("rank", C.c_int32), ("outer_iters", C.c_int32),
        ("inner_iters", C.c_int32), ("status", C.c_int32), ("kernel_launches", C.c_int64),
        ("admm_iters", C.c_int32), ("cg_steps", C.c_int32), ("reopt_rounds", C.c_int32),
        ("reserved_r", C.c_int32), ("reopt_scale", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class lorads_batch_shape(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("rows_per_warp", C.c_int32), ("order", C.c_int32),
                ("threads", C.c_int32), ("cluster", C.c_int32), ("team_count", C.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class lorads_batch_stats(C.Structure):
    _fields_ = [
        ("seconds", C.c_double), ("instances_per_s", C.c_double), ("latency_p50_ms", C.c_double),
        ("latency_p99_ms", C.c_double), ("latency_max_ms", C.c_double), ("inner_iters", C.c_int64),
        ("solved", C.c_int32), ("grid", C.c_int32), ("shape", lorads_batch_shape),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "shape"}
        d["shape"] = self.shape.as_dict()
        return d


_VP, _DP, _I64P, _I32P = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "lorads_default_params": (None, [C.POINTER(lorads_params)]),
    "lorads_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, _I64P, _I32P, _DP, C.c_int64, C.c_int64,
                                _I32P, _I32P, _I32P, _DP, _DP, C.POINTER(lorads_params), C.c_void_p]),
    "lorads_spmm": (C.c_int, [_VP, _VP, C.c_int32, C.c_int32, _VP, _VP, C.c_int32]),
    "lorads_constraint_eval": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_int32, _VP, C.c_int32]),
    "lorads_linesearch_coeffs": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_int32, _VP, C.c_double, _DP, _DP,
                                           C.c_int32]),
    "lorads_solve": (C.c_int, [_VP, _VP, C.c_int32, C.c_int32, _VP, C.POINTER(lorads_result)]),
    "lorads_get_solution": (C.c_int, [_VP, _DP, C.c_int64, _I32P, _DP]),
    "lorads_last_error": (C.c_char_p, [_VP]),
    "lorads_create_error": (C.c_char_p, []),
    "lorads_destroy": (None, [_VP]),
    "lorads_problem_info": (C.c_int, [_VP, _I64P, _I64P, _I64P, _I64P, _I64P]),
    "lorads_kernel_times": (C.c_int32, [_VP, C.POINTER(C.c_char_p), _DP, C.c_int32]),
    "lorads_kernel_counts": (C.c_int32, [_VP, C.POINTER(C.c_char_p), _I64P, C.c_int32]),
    "lorads_set_iteration_limit": (C.c_int, [_VP, C.c_int64]),
    "lorads_linesearch_coeffs_noalloc": (C.c_int, [C.c_int64, _VP, _VP, _VP, C.c_int64, _VP, _VP, _VP, _VP, _VP,
                                                   _VP, _VP, C.c_int32, C.c_int32, _VP, C.c_double, _VP, _VP]),
    "lorads_noalloc_error": (C.c_char_p, []),
    "lorads_dual_min_eig": (C.c_int, [_VP, _VP, C.c_int32, C.c_uint64, _DP]),
    "lorads_admm_operator": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_int32, C.c_double, _VP, C.c_int32]),
    "lorads_admm_cg": (C.c_int, [_VP, _VP, _VP, _VP, C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                 _I32P, C.c_int32]),
    "lorads_admm_stage": (C.c_int, [_VP, _VP, C.c_int32, C.c_int32, _VP, C.c_double, C.POINTER(lorads_result)]),
    "lorads_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, _I64P, _I64P, _I64P, _I32P, _DP, _I32P,
                                      _I32P, _I32P, _DP, _DP, _I32P, _DP, C.POINTER(lorads_params), C.c_void_p]),
    "lorads_batch_solve": (C.c_int, [_VP, C.POINTER(lorads_result), C.POINTER(lorads_batch_stats)]),
    "lorads_batch_tune": (C.c_int, [_VP, C.c_int32, C.POINTER(lorads_batch_shape)]),
    "lorads_batch_set_shape": (C.c_int, [_VP, C.POINTER(lorads_batch_shape)]),
    "lorads_batch_set_iteration_limit": (C.c_int, [_VP, C.c_int64]),
    "lorads_batch_get_solution": (C.c_int, [_VP, C.c_int32, _DP, C.c_int64, _I32P, _DP]),
    "lorads_batch_create_error": (C.c_char_p, []),
    "lorads_batch_phase_times": (C.c_int32, [_VP, C.c_int32, C.POINTER(C.c_char_p), _DP, C.c_int32]),
    "lorads_batch_last_error": (C.c_char_p, [_VP]),
    "lorads_batch_destroy": (None, [_VP]),
    "lorads_gnn_param_count": (C.c_int64, [C.c_int32]),
    "lorads_gnn_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.POINTER(C.c_float), C.c_void_p]),
    "lorads_gnn_get_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int64]),
    "lorads_gnn_set_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int64]),
    "lorads_gnn_predict": (C.c_int, [_VP, C.c_int64, _VP, _VP, _VP, C.c_uint64, C.c_int32, _VP]),
    "lorads_gnn_edge_targets": (C.c_int, [C.c_int64, _VP, _VP, _VP, C.c_int32, C.c_int32, _VP, _VP]),
    "lorads_gnn_train_step": (C.c_int, [_VP, C.c_int64, _VP, _VP, _VP, C.c_uint64, _VP, C.c_int64, C.c_float, _DP,
                                        _VP]),
    "lorads_gnn_last_error": (C.c_char_p, [_VP]),
    "lorads_gnn_create_error": (C.c_char_p, []),
    "lorads_gnn_destroy": (None, [_VP]),
}

_lib = None


def load(path: str | os.PathLike | None = None) -> C.CDLL:
    """Loads liblorads.so (raises when it is missing: build it with builder.py)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise ImportError(f"{p} not found: build the CUDA library first "
                          "(python paper_2407_15049_gb300/builder.py)")
    lib = C.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def default_params(**overrides) -> lorads_params:
    p = lorads_params()
    load().lorads_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _check(ctx, status: int):
    if status != LORADS_OK:
        msg = load().lorads_last_error(ctx).decode() if ctx else ""
        raise LoradsError(status, msg)


def _dptr(t) -> int:
    """Device address of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _prec_of(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return LORADS_FP64
    if t.dtype == torch.float32:
        return LORADS_FP32
    if t.dtype == torch.bfloat16:
        return LORADS_BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def lorads_create(inst, params: lorads_params | None = None, stream: int | None = None) -> C.c_void_p:
    """Uploads an SDP instance (object with n, rowptr, colind, val, m, con, row, col, aval, b)."""
    lib = load()
    rowptr = np.ascontiguousarray(inst.rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(inst.colind, dtype=np.int32)
    val = np.ascontiguousarray(inst.val, dtype=np.float64)
    con = np.ascontiguousarray(inst.con, dtype=np.int32)
    row = np.ascontiguousarray(inst.row, dtype=np.int32)
    col = np.ascontiguousarray(inst.col, dtype=np.int32)
    aval = np.ascontiguousarray(inst.aval, dtype=np.float64)
    b = np.ascontiguousarray(inst.b, dtype=np.float64)
    ctx = C.c_void_p()
    st = lib.lorads_create(C.byref(ctx), int(inst.n), _ptr(rowptr, C.c_int64), _ptr(colind, C.c_int32),
                           _ptr(val, C.c_double), int(inst.m), int(len(con)), _ptr(con, C.c_int32),
                           _ptr(row, C.c_int32), _ptr(col, C.c_int32), _ptr(aval, C.c_double),
                           _ptr(b, C.c_double), C.byref(params) if params is not None else None,
                           C.c_void_p(stream) if stream else None)
    if st != LORADS_OK:
        raise LoradsError(st, lib.lorads_create_error().decode())
    return ctx


def lorads_destroy(ctx) -> None:
    if ctx:
        load().lorads_destroy(ctx)


def lorads_spmm(ctx, R, v, out, r: int | None = None) -> None:
    """out = (C - A*(v)) R on device tensors (R, out: n x ld; v: float64[m] or None)."""
    ld = R.shape[1]
    _check(ctx, load().lorads_spmm(ctx, _dptr(R), int(r or ld), int(ld), _dptr(v), _dptr(out), _prec_of(R)))


def lorads_constraint_eval(ctx, U, V, out, r: int | None = None) -> None:
    """out_k = <A_k, U V^T> (out: float64[m] device tensor)."""
    ld = U.shape[1]
    _check(ctx, load().lorads_constraint_eval(ctx, _dptr(U), _dptr(V), int(r or ld), int(ld), _dptr(out),
                                              _prec_of(U)))


def lorads_linesearch_coeffs(ctx, R, D, y, rho: float, r: int | None = None):
    """Returns (a[4] as numpy, tau)."""
    ld = R.shape[1]
    a = np.zeros(4)
    tau = C.c_double()
    _check(ctx, load().lorads_linesearch_coeffs(ctx, _dptr(R), _dptr(D), int(r or ld), int(ld), _dptr(y),
                                                float(rho), _ptr(a, C.c_double), C.byref(tau), _prec_of(R)))
    return a, tau.value


def lorads_solve(ctx, R0=None, y0: np.ndarray | None = None, r0: int = 0, on_device: bool = False,
                 raise_on_status: bool = False, max_total_inner: int = 0) -> dict:
    """Runs the solver.  R0: host numpy (n x r0) or device float64 tensor, or None.
    max_total_inner > 0 stops after that many L-BFGS iterations in total."""
    lib = load()
    res = lorads_result()
    keep = []
    if R0 is None:
        rp, r0v, dev = None, int(r0), 0
    elif on_device or not isinstance(R0, np.ndarray):
        rp, r0v, dev = C.c_void_p(_dptr(R0)), int(R0.shape[1]), 1
    else:
        R0 = np.ascontiguousarray(R0, dtype=np.float64)
        keep.append(R0)
        rp, r0v, dev = C.c_void_p(R0.ctypes.data), int(R0.shape[1]), 0
    yp = None
    if y0 is not None:
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        keep.append(y0)
        yp = C.c_void_p(y0.ctypes.data)
    if max_total_inner:
        _check(ctx, lib.lorads_set_iteration_limit(ctx, int(max_total_inner)))
    st = lib.lorads_solve(ctx, rp, r0v, dev, yp, C.byref(res))
    if max_total_inner:
        _check(ctx, lib.lorads_set_iteration_limit(ctx, 0))
    out = res.as_dict()
    out["status_name"] = STATUS_NAMES.get(res.status, str(res.status))
    if st not in (LORADS_OK, 5, 6, 7) or (raise_on_status and st != LORADS_OK):
        _check(ctx, st)
    return out


def lorads_admm_operator(ctx, V, X, out, rho: float, r: int | None = None) -> None:
    """out = rho A*(A(X V^T)) V + rho X on device tensors (n x ld, float64 or float32)."""
    ld = V.shape[1]
    _check(ctx, load().lorads_admm_operator(ctx, _dptr(V), _dptr(X), int(r or ld), int(ld), float(rho), _dptr(out),
                                            _prec_of(V)))


def lorads_admm_cg(ctx, V, X, y, rho: float, cg_rel: float = 1e-2, cg_max: int = 50, r: int | None = None) -> int:
    """Solves rho A*(A(X V^T)) V + rho X = -C V + A*(y) V + rho A*(b) V + rho V by CG in
    place from X; returns the number of CG steps."""
    ld = V.shape[1]
    steps = C.c_int32()
    _check(ctx, load().lorads_admm_cg(ctx, _dptr(V), _dptr(X), _dptr(y), float(rho), int(r or ld), int(ld),
                                      float(cg_rel), int(cg_max), C.byref(steps), _prec_of(V)))
    return steps.value


def lorads_admm_stage(ctx, R0, y0: np.ndarray | None, rho: float, on_device: bool = False) -> dict:
    """Runs the ADMM stage alone from U = V = R0, multiplier y0 and penalty rho."""
    lib = load()
    res = lorads_result()
    keep = []
    if on_device or not isinstance(R0, np.ndarray):
        rp, r0v, dev = C.c_void_p(_dptr(R0)), int(R0.shape[1]), 1
    else:
        R0 = np.ascontiguousarray(R0, dtype=np.float64)
        keep.append(R0)
        rp, r0v, dev = C.c_void_p(R0.ctypes.data), int(R0.shape[1]), 0
    yp = None
    if y0 is not None:
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        keep.append(y0)
        yp = C.c_void_p(y0.ctypes.data)
    st = lib.lorads_admm_stage(ctx, rp, r0v, dev, yp, float(rho), C.byref(res))
    out = res.as_dict()
    out["status_name"] = STATUS_NAMES.get(res.status, str(res.status))
    if st not in (LORADS_OK, 5, 6, 7):
        _check(ctx, st)
    return out


def lorads_get_solution(ctx, n: int, m: int):
    """Returns (R as numpy n x rank, y as numpy m)."""
    lib = load()
    rank = C.c_int32()
    _check(ctx, lib.lorads_get_solution(ctx, None, 0, C.byref(rank), None))
    R = np.zeros((n, rank.value))
    y = np.zeros(m)
    _check(ctx, lib.lorads_get_solution(ctx, _ptr(R, C.c_double), R.size, C.byref(rank), _ptr(y, C.c_double)))
    return R, y


def lorads_dual_min_eig(ctx, y=None, steps: int = 200, seed: int = 1) -> float:
    """sigma_min(C - A*(y)) by Lanczos on the GPU (y: device float64[m] or None)."""
    out = C.c_double()
    _check(ctx, load().lorads_dual_min_eig(ctx, _dptr(y), int(steps), int(seed), C.byref(out)))
    return out.value


def lorads_problem_info(ctx) -> dict:
    vals = [C.c_int64() for _ in range(5)]
    _check(ctx, load().lorads_problem_info(ctx, *[C.byref(v) for v in vals]))
    return dict(zip(["n", "m", "nnz_c", "m_diag", "m_offdiag"], [v.value for v in vals]))


def lorads_kernel_times(ctx) -> dict:
    """{kernel family: (average ms, launches)} of the last profiled (verbose >= 2) solve."""
    lib = load()
    names = (C.c_char_p * 32)()
    ms = (C.c_double * 32)()
    counts = (C.c_int64 * 32)()
    k = lib.lorads_kernel_times(ctx, names, ms, 32)
    lib.lorads_kernel_counts(ctx, names, counts, 32)
    return {names[i].decode(): (ms[i], counts[i]) for i in range(k)}


def padded_ld(r: int) -> int:
    """Row width the kernels use for rank r (r rounded up to a multiple of 4)."""
    return (int(r) + 3) // 4 * 4


# ------------------------------------------------------------------ batched solve
def _bcheck(batch, status: int):
    if status != LORADS_OK:
        raise LoradsError(status, load().lorads_batch_last_error(batch).decode() if batch else "")


def lorads_batch_create(instances, params: lorads_params | None = None, r0=None, R0=None,
                        stream: int | None = None) -> C.c_void_p:
    """Uploads a list of SDP instances (objects as for lorads_create) as one batch.
    r0: per-instance starting ranks or None; R0: list of n_i x r0_i float64 arrays or None."""
    lib = load()
    cat = lambda key, dt: np.ascontiguousarray(  # noqa: E731
        np.concatenate([np.asarray(getattr(t, key), dtype=dt) for t in instances]), dtype=dt)
    n = np.array([t.n for t in instances], dtype=np.int64)
    m = np.array([t.m for t in instances], dtype=np.int64)
    rowptr, colind, val = cat("rowptr", np.int64), cat("colind", np.int32), cat("val", np.float64)
    con, row, col = cat("con", np.int32), cat("row", np.int32), cat("col", np.int32)
    aval, b = cat("aval", np.float64), cat("b", np.float64)
    r0a = None if r0 is None else np.ascontiguousarray(r0, dtype=np.int32)
    R0a = None
    if R0 is not None:
        R0a = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in R0]))
        if r0a is None:
            r0a = np.array([np.asarray(x).shape[1] for x in R0], dtype=np.int32)
    out = C.c_void_p()
    st = lib.lorads_batch_create(
        C.byref(out), len(instances), _ptr(n, C.c_int64), _ptr(m, C.c_int64), _ptr(rowptr, C.c_int64),
        _ptr(colind, C.c_int32), _ptr(val, C.c_double), _ptr(con, C.c_int32), _ptr(row, C.c_int32),
        _ptr(col, C.c_int32), _ptr(aval, C.c_double), _ptr(b, C.c_double),
        _ptr(r0a, C.c_int32) if r0a is not None else None, _ptr(R0a, C.c_double) if R0a is not None else None,
        C.byref(params) if params is not None else None, C.c_void_p(stream) if stream else None)
    if st != LORADS_OK:
        raise LoradsError(st, lib.lorads_batch_create_error().decode())
    return out


def lorads_batch_solve(batch, count: int, max_total_inner: int = 0):
    """Solves every instance in one persistent launch.  Returns (list of result dicts, stats dict)."""
    lib = load()
    if max_total_inner:
        _bcheck(batch, lib.lorads_batch_set_iteration_limit(batch, int(max_total_inner)))
    res = (lorads_result * count)()
    stats = lorads_batch_stats()
    st = lib.lorads_batch_solve(batch, res, C.byref(stats))
    if max_total_inner:
        _bcheck(batch, lib.lorads_batch_set_iteration_limit(batch, 0))
    _bcheck(batch, st)
    out = []
    for r in res:
        d = r.as_dict()
        d["status_name"] = STATUS_NAMES.get(r.status, str(r.status))
        out.append(d)
    return out, stats.as_dict()


def lorads_batch_tune(batch, probe_iters: int = 30) -> dict:
    shape = lorads_batch_shape()
    _bcheck(batch, load().lorads_batch_tune(batch, int(probe_iters), C.byref(shape)))
    return shape.as_dict()


def lorads_batch_set_shape(batch, ctas_per_sm: int, rows_per_warp: int, order: int, threads: int = 256,
                           cluster: int = 1, team_count: int = 0) -> None:
    shape = lorads_batch_shape(int(ctas_per_sm), int(rows_per_warp), int(order), int(threads), int(cluster),
                               int(team_count))
    _bcheck(batch, load().lorads_batch_set_shape(batch, C.byref(shape)))


def lorads_batch_get_solution(batch, i: int, n: int, m: int):
    """Returns (R as numpy n x rank, y as numpy m) of instance i."""
    lib = load()
    rank = C.c_int32()
    _bcheck(batch, lib.lorads_batch_get_solution(batch, int(i), None, 0, C.byref(rank), None))
    R = np.zeros((n, rank.value))
    y = np.zeros(m)
    _bcheck(batch, lib.lorads_batch_get_solution(batch, int(i), _ptr(R, C.c_double), R.size, C.byref(rank),
                                                 _ptr(y, C.c_double)))
    return R, y


def lorads_batch_phase_times(batch, i: int = -1) -> dict:
    """{phase: ms} of instance i's solve in the last launch (i = -1: all instances)."""
    names = (C.c_char_p * 16)()
    ms = (C.c_double * 16)()
    k = load().lorads_batch_phase_times(batch, int(i), names, ms, 16)
    return {names[q].decode(): ms[q] for q in range(k)}


def lorads_batch_destroy(batch) -> None:
    if batch:
        load().lorads_batch_destroy(batch)


# ------------------------------------------------------------------ learned warm start
def _gcheck(net, status: int):
    if status != LORADS_OK:
        raise LoradsError(status, load().lorads_gnn_last_error(net).decode() if net else "")


def lorads_gnn_param_count(r_out: int) -> int:
    return int(load().lorads_gnn_param_count(int(r_out)))


def lorads_gnn_create(r_out: int, theta0: np.ndarray, act_prec: int = LORADS_BF16,
                      stream: int | None = None) -> C.c_void_p:
    lib = load()
    th = np.ascontiguousarray(theta0, dtype=np.float32)
    if th.size != lorads_gnn_param_count(r_out):
        raise ValueError("theta0 has the wrong size")
    out = C.c_void_p()
    st = lib.lorads_gnn_create(C.byref(out), int(r_out), int(act_prec), _ptr(th, C.c_float),
                               C.c_void_p(stream) if stream else None)
    if st != LORADS_OK:
        raise LoradsError(st, lib.lorads_gnn_create_error().decode())
    return out


def lorads_gnn_get_params(net, r_out: int) -> np.ndarray:
    th = np.zeros(lorads_gnn_param_count(r_out), dtype=np.float32)
    _gcheck(net, load().lorads_gnn_get_params(net, _ptr(th, C.c_float), th.size))
    return th


def lorads_gnn_set_params(net, theta: np.ndarray) -> None:
    th = np.ascontiguousarray(theta, dtype=np.float32)
    _gcheck(net, load().lorads_gnn_set_params(net, _ptr(th, C.c_float), th.size))


def lorads_gnn_predict(net, graph: dict, feature_seed: int, R_out, ld: int) -> None:
    """graph: dict with n and device tensors rowptr (int64), colind (int32), val (float64)."""
    _gcheck(net, load().lorads_gnn_predict(net, int(graph["n"]), _dptr(graph["rowptr"]), _dptr(graph["colind"]),
                                           _dptr(graph["val"]), int(feature_seed), int(ld), _dptr(R_out)))


def lorads_gnn_edge_targets(graph: dict, R, r: int, ld: int, targets, stream: int | None = None) -> None:
    st = load().lorads_gnn_edge_targets(int(graph["n"]), _dptr(graph["rowptr"]), _dptr(graph["colind"]), _dptr(R),
                                        int(r), int(ld), _dptr(targets), C.c_void_p(stream) if stream else None)
    if st != LORADS_OK:
        raise LoradsError(st, "lorads_gnn_edge_targets")


def lorads_gnn_train_step(net, graph: dict, feature_seed: int, targets, lr: float, grad_out=None,
                          want_loss: bool = True):
    loss = C.c_double()
    _gcheck(net, load().lorads_gnn_train_step(net, int(graph["n"]), _dptr(graph["rowptr"]), _dptr(graph["colind"]),
                                              _dptr(graph["val"]), int(feature_seed), _dptr(targets),
                                              int(graph["n_edges"]), float(lr),
                                              C.byref(loss) if want_loss else None, _dptr(grad_out)))
    return loss.value if want_loss else None


def lorads_gnn_destroy(net) -> None:
    if net:
        load().lorads_gnn_destroy(net)

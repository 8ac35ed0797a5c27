"""Thin ctypes binding of libpdlp.so (include/pdlp.h): argument marshalling only.

Arrays are numpy (host) or torch CUDA tensors (device); every computation happens in
the library's CUDA kernels.  There is no CPU fallback: if the shared library is
missing, loading fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdlp.so")

TRACE_HEADER = 8
STATUS_NAMES = {0: "OPTIMAL", 1: "ITERATION_LIMIT", 2: "TIME_LIMIT", 3: "PRIMAL_INFEASIBLE",
                4: "DUAL_INFEASIBLE", 5: "NUMERICAL_ERROR", -1: "INVALID_ARGUMENT",
                -2: "OUT_OF_MEMORY", -3: "CUDA_ERROR"}
FP64, FP32_BULK = 0, 1
POLISH_LOG_COLS = 7   # PDLP_POLISH_LOG_COLS
POLISH_LOG_CAP = 64   # pauses recorded per solve (k = 100 * 2^63 is never reached)


class Csr(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [
        ("eps_rel_kkt", ctypes.c_double), ("termination_mode", ctypes.c_int),
        ("eps_abs_feas", ctypes.c_double), ("eps_rel_gap", ctypes.c_double),
        ("max_iters", ctypes.c_int64), ("time_limit_s", ctypes.c_double),
        ("ruiz_iters", ctypes.c_int), ("pc_alpha", ctypes.c_double),
        ("check_period", ctypes.c_int), ("beta_suff", ctypes.c_double),
        ("beta_nec", ctypes.c_double), ("beta_art", ctypes.c_double),
        ("theta", ctypes.c_double), ("eps_zero", ctypes.c_double),
        ("max_step_retries", ctypes.c_int), ("precision", ctypes.c_int),
        ("inputs_on_device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
        ("trace_iters", ctypes.c_int64), ("trace_out", ctypes.c_void_p),
        ("profile", ctypes.c_int), ("verbose", ctypes.c_int),
        ("feasibility_polishing", ctypes.c_int), ("polish_log_cap", ctypes.c_int64),
        ("polish_log", ctypes.c_void_p),
        ("detect_infeasibility", ctypes.c_int), ("eps_infeas", ctypes.c_double),
        ("reduced_costs", ctypes.c_int),
        ("fixed_step", ctypes.c_double), ("fixed_omega", ctypes.c_double),
    ]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", Csr),
                ("c", ctypes.c_void_p), ("lc", ctypes.c_void_p), ("uc", ctypes.c_void_p),
                ("lv", ctypes.c_void_p), ("uv", ctypes.c_void_p),
                ("x_out", ctypes.c_void_p), ("y_out", ctypes.c_void_p)]


class UnrolledProblem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", Csr),
                ("c", ctypes.c_void_p), ("lc", ctypes.c_void_p), ("uc", ctypes.c_void_p),
                ("lv", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("K", ctypes.c_int64),
                ("eta", ctypes.c_double), ("omega", ctypes.c_double),
                ("checkpoint_every", ctypes.c_int64), ("gx", ctypes.c_void_p),
                ("gy", ctypes.c_void_p), ("x_out", ctypes.c_void_p), ("y_out", ctypes.c_void_p),
                ("grad_c", ctypes.c_void_p), ("grad_lc", ctypes.c_void_p),
                ("grad_uc", ctypes.c_void_p), ("grad_lv", ctypes.c_void_p),
                ("grad_uv", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int64), ("attempts", ctypes.c_int64),
        ("rejected_steps", ctypes.c_int64), ("restarts", ctypes.c_int64 * 3),
        ("kkt_passes", ctypes.c_double),
        ("rel_kkt", ctypes.c_double), ("rel_primal", ctypes.c_double),
        ("rel_dual", ctypes.c_double), ("rel_gap", ctypes.c_double),
        ("primal_res_l2", ctypes.c_double), ("dual_res_l2", ctypes.c_double),
        ("primal_res_inf", ctypes.c_double), ("dual_res_inf", ctypes.c_double),
        ("pobj", ctypes.c_double), ("dobj", ctypes.c_double), ("paper_gap", ctypes.c_double),
        ("omega", ctypes.c_double), ("eta_hat", ctypes.c_double),
        ("seconds_setup", ctypes.c_double), ("seconds_solve", ctypes.c_double),
        ("seconds_total", ctypes.c_double),
        ("ms_spmv_a", ctypes.c_double), ("ms_spmv_at", ctypes.c_double),
        ("ms_primal", ctypes.c_double), ("ms_checks", ctypes.c_double),
        ("launches_spmv_a", ctypes.c_int64), ("launches_spmv_at", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("bytes_spmv_a", ctypes.c_double), ("bytes_spmv_at", ctypes.c_double),
        ("gap_evals", ctypes.c_int64), ("gap_fallbacks", ctypes.c_int64),
        ("gap_failures", ctypes.c_int64),
        ("polish_pauses", ctypes.c_int64), ("polish_primal_iters", ctypes.c_int64),
        ("polish_dual_iters", ctypes.c_int64), ("polish_accepted_k", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("ms_gap", ctypes.c_double), ("ms_kkt", ctypes.c_double), ("ms_infeas", ctypes.c_double),
        ("evaluations", ctypes.c_int64),
        ("primal_res_rel_inf", ctypes.c_double), ("dual_res_rel_inf", ctypes.c_double),
        ("batch_launch_s", ctypes.c_double), ("batch_sm", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "restarts" else v
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_lib = None


def load_library(path: str | None = None):
    """Loads libpdlp.so once and declares the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.pdlp_params_default.argtypes = [ctypes.POINTER(Params)]
    lib.pdlp_params_default.restype = None
    lib.pdlp_last_error.argtypes = []
    lib.pdlp_last_error.restype = ctypes.c_char_p
    lib.pdlp_solve.argtypes = [i64, i64, ctypes.POINTER(Csr), P, P, P, P, P,
                               ctypes.POINTER(Params), P, P, ctypes.POINTER(Stats)]
    lib.pdlp_solve.restype = ctypes.c_int
    lib.pdlp_precondition.argtypes = [i64, i64, ctypes.POINTER(Csr), ctypes.POINTER(Params),
                                      P, P, P]
    lib.pdlp_precondition.restype = ctypes.c_int
    lib.pdlp_normalized_gap.argtypes = [i64, i64, ctypes.POINTER(Csr), P, P, P, P, P, P, P, P, P,
                                        ctypes.c_double, ctypes.POINTER(Params),
                                        ctypes.POINTER(ctypes.c_double)]
    lib.pdlp_normalized_gap.restype = ctypes.c_int
    lib.pdlp_kkt.argtypes = [i64, i64, ctypes.POINTER(Csr), P, P, P, P, P, P, P,
                             ctypes.POINTER(Params), P]
    lib.pdlp_kkt.restype = ctypes.c_int
    lib.pdlp_kkt_products_noalloc.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P, P, P]
    lib.pdlp_kkt_products_noalloc.restype = ctypes.c_int
    lib.pdlp_solve_batch.argtypes = [i64, P, ctypes.POINTER(Params), ctypes.c_int, P, P]
    lib.pdlp_solve_batch.restype = ctypes.c_int
    lib.pdlp_solve_batch_persistent.argtypes = [i64, P, ctypes.POINTER(Params), ctypes.c_int, P,
                                                P, P]
    lib.pdlp_solve_batch_persistent.restype = ctypes.c_int
    lib.pdlp_unrolled_pdhg.argtypes = [i64, i64, ctypes.POINTER(Csr), P, P, P, P, P, i64,
                                       ctypes.c_double, ctypes.c_double, i64, P, P,
                                       ctypes.POINTER(Params), P, P, P, P, P, P, P]
    lib.pdlp_unrolled_pdhg.restype = ctypes.c_int
    lib.pdlp_unrolled_pdhg_batch.argtypes = [i64, P, ctypes.POINTER(Params), ctypes.c_int, P]
    lib.pdlp_unrolled_pdhg_batch_persistent.argtypes = [i64, P, ctypes.POINTER(Params), P]
    lib.pdlp_unrolled_pdhg_batch_persistent.restype = ctypes.c_int
    lib.pdlp_gather_bench.argtypes = [ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, i64,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, P]
    lib.pdlp_gather_bench.restype = ctypes.c_int
    lib.pdlp_unrolled_pdhg_batch.restype = ctypes.c_int
    _lib = lib
    return lib


class PdlpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def default_params(**overrides) -> Params:
    lib = load_library()
    p = Params()
    lib.pdlp_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# array marshalling: numpy on the host, torch tensors on the device
# ---------------------------------------------------------------------------
def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _host(a, dtype):
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return arr, arr.ctypes.data


def _dev(a, torch_dtype):
    t = a.contiguous()
    if t.dtype != torch_dtype:
        t = t.to(torch_dtype)
    return t, t.data_ptr()


class _Marshal:
    def __init__(self, on_device: bool):
        self.on_device = on_device
        self.keep = []
        if on_device:
            import torch

            self.torch = torch

    def __call__(self, a, kind):
        if a is None:
            return None
        if self.on_device:
            tdt = {"f64": self.torch.float64, "i64": self.torch.int64, "i32": self.torch.int32}[kind]
            t, p = _dev(a, tdt)
        else:
            ndt = {"f64": np.float64, "i64": np.int64, "i32": np.int32}[kind]
            t, p = _host(a, ndt)
        self.keep.append(t)
        return p

    def out(self, n):
        if self.on_device:
            t = self.torch.empty(max(n, 0), dtype=self.torch.float64, device="cuda")
            return t, t.data_ptr() if n > 0 else None
        arr = np.empty(max(n, 0))
        return arr, arr.ctypes.data if n > 0 else None


def _check(code):
    if code < 0:
        raise PdlpError(code, load_library().pdlp_last_error().decode())
    return code


@dataclasses.dataclass
class SolveResult:
    status: int
    x: object
    y: object
    stats: dict
    trace: list

    @property
    def status_name(self):
        return STATUS_NAMES.get(self.status, str(self.status))


def _params_for(on_device: bool, params: dict):
    prm = default_params(**params)
    prm.inputs_on_device = 1 if on_device else 0
    if on_device and not params.get("cuda_stream"):
        import torch

        prm.cuda_stream = torch.cuda.current_stream().cuda_stream
    return prm


def _lp_args(mh, m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv):
    A = Csr()
    A.nnz = int(len(val)) if not hasattr(val, "numel") else int(val.numel())
    A.row_ptr = mh(row_ptr, "i64")
    A.col_idx = mh(col_idx, "i32")
    A.val = mh(val, "f64")
    vecs = [mh(c, "f64"), mh(lc, "f64"), mh(uc, "f64"), mh(lv, "f64"), mh(uv, "f64")]
    return A, vecs


def solve(m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv, trace_iters: int = 0,
          **params) -> SolveResult:
    """pdlp_solve.  Inputs are numpy arrays (host) or torch CUDA tensors (device; then
    x and y come back as CUDA tensors).  ``params`` are pdlp_params fields."""
    lib = load_library()
    on_device = _is_cuda_tensor(val) or _is_cuda_tensor(c)
    mh = _Marshal(on_device)
    A, vecs = _lp_args(mh, m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv)
    prm = _params_for(on_device, params)
    trace_buf = None
    if trace_iters > 0:
        trace_buf = np.full((trace_iters, TRACE_HEADER + n + m), np.nan)
        prm.trace_iters = trace_iters
        prm.trace_out = trace_buf.ctypes.data
    log_buf = None
    if prm.feasibility_polishing:
        log_buf = np.zeros((POLISH_LOG_CAP, POLISH_LOG_COLS))
        prm.polish_log_cap = POLISH_LOG_CAP
        prm.polish_log = log_buf.ctypes.data
    x, xp = mh.out(n)
    y, yp = mh.out(m)
    st = Stats()
    code = lib.pdlp_solve(m, n, ctypes.byref(A), *vecs, ctypes.byref(prm), xp, yp, ctypes.byref(st))
    _check(code)
    stats = st.as_dict()
    if log_buf is not None:
        rows = log_buf[:min(stats["polish_pauses"], POLISH_LOG_CAP)]
        stats["polish"] = [dict(k=int(r[0]), paper_gap=r[1], primal_iters=int(r[2]),
                                primal_ok=bool(r[3]), dual_iters=int(r[4]), dual_ok=bool(r[5]),
                                accepted=bool(r[6])) for r in rows]
    if stats["gap_failures"]:
        stats["gap_failure_message"] = lib.pdlp_last_error().decode()
    trace = []
    if trace_buf is not None:
        for row in trace_buf:
            if not (row[0] >= 1):
                break
            trace.append(dict(k=int(row[0]), eta=row[1], omega=row[2], eta_hat=row[3],
                              attempts=int(row[4]), restart=int(row[5]), mu_cur=row[6],
                              mu_avg=row[7], x=row[TRACE_HEADER:TRACE_HEADER + n].copy(),
                              y=row[TRACE_HEADER + n:].copy()))
    return SolveResult(code, x, y, stats, trace)


def solve_instance(inst, trace_iters: int = 0, device: bool = False, **params) -> SolveResult:
    """Convenience wrapper for an object with m, n, row_ptr, col_idx, val, c, lc, uc,
    lv, uv attributes; ``device=True`` stages the arrays as CUDA tensors first."""
    arrs = [inst.row_ptr, inst.col_idx, inst.val, inst.c, inst.lc, inst.uc, inst.lv, inst.uv]
    if device:
        import torch

        arrs = [torch.as_tensor(np.asarray(a)).cuda() for a in arrs]
    return solve(inst.m, inst.n, *arrs, trace_iters=trace_iters, **params)


def solve_batch(instances, device: bool = False, concurrency: int = 16, persistent: bool = False,
                tune: int = 0, **params) -> list:
    """pdlp_solve_batch over objects with m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv
    attributes (host arrays; ``device=True`` stages them as CUDA tensors first).
    ``persistent=True`` calls pdlp_solve_batch_persistent instead (one launch for the
    whole batch; ``tune`` as there, the configuration used lands in every result's
    ``stats['tune']``).  Returns one SolveResult per instance, in order; a negative
    status does not raise (its message is in ``stats['error']`` of the first failing
    instance)."""
    lib = load_library()
    mh = _Marshal(device)
    probs = (Problem * max(1, len(instances)))()
    outs = []
    for k, inst in enumerate(instances):
        arrs = [inst.row_ptr, inst.col_idx, inst.val, inst.c, inst.lc, inst.uc, inst.lv, inst.uv]
        if device:
            import torch

            arrs = [torch.as_tensor(np.asarray(a)).cuda() for a in arrs]
        A, vecs = _lp_args(mh, inst.m, inst.n, *arrs)
        x, xp = mh.out(inst.n)
        y, yp = mh.out(inst.m)
        pr = probs[k]
        pr.m, pr.n, pr.A = inst.m, inst.n, A
        pr.c, pr.lc, pr.uc, pr.lv, pr.uv = vecs
        pr.x_out, pr.y_out = xp, yp
        outs.append((x, y))
    prm = _params_for(device, params)
    status = (ctypes.c_int * max(1, len(instances)))()
    stats = (Stats * max(1, len(instances)))()
    tune_used = ctypes.c_int(0)
    if persistent:
        _check(lib.pdlp_solve_batch_persistent(len(instances), ctypes.addressof(probs),
                                               ctypes.byref(prm), int(tune),
                                               ctypes.addressof(status), ctypes.addressof(stats),
                                               ctypes.addressof(tune_used)))
    else:
        _check(lib.pdlp_solve_batch(len(instances), ctypes.addressof(probs), ctypes.byref(prm),
                                    int(concurrency), ctypes.addressof(status),
                                    ctypes.addressof(stats)))
    res = []
    first_error = lib.pdlp_last_error().decode()
    for k, (x, y) in enumerate(outs):
        st = stats[k].as_dict()
        if persistent:
            st["tune"] = tune_used.value
        if status[k] < 0 and first_error:
            st["error"] = first_error
            first_error = ""
        res.append(SolveResult(status[k], x, y, st, []))
    return res


GRAD_KEYS = ("c", "lc", "uc", "lv", "uv")


def unrolled_pdhg(m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv, K, eta, omega, gx=None,
                  gy=None, checkpoint_every=50, **params):
    """pdlp_unrolled_pdhg: (x_K, y_K) of K fixed-step PDHG steps and, when gx, gy are
    given, the gradients of gx'x_K + gy'y_K with respect to c, lc, uc, lv, uv (dict).
    Arrays are numpy (host) or torch CUDA tensors (device), outputs alike."""
    lib = load_library()
    on_device = _is_cuda_tensor(val) or _is_cuda_tensor(c)
    mh = _Marshal(on_device)
    A, vecs = _lp_args(mh, m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv)
    prm = _params_for(on_device, params)
    x, xp = mh.out(n)
    y, yp = mh.out(m)
    want = gx is not None
    gptr = [mh(gx, "f64"), mh(gy, "f64")] if want else [None, None]
    grads, gouts = {}, []
    for k, ln in zip(GRAD_KEYS, (n, m, m, n, n)):
        if want:
            t, p_ = mh.out(ln)
            grads[k] = t
            gouts.append(p_)
        else:
            gouts.append(None)
    _check(lib.pdlp_unrolled_pdhg(m, n, ctypes.byref(A), *vecs, int(K), float(eta), float(omega),
                                  int(checkpoint_every), *gptr, ctypes.byref(prm), xp, yp, *gouts))
    return x, y, (grads if want else None)


def unrolled_pdhg_batch(items, device: bool = False, concurrency: int = 16,
                        persistent: bool = False, **params) -> list:
    """pdlp_unrolled_pdhg_batch (``persistent=True``: pdlp_unrolled_pdhg_batch_persistent,
    one launch for the whole batch).  ``items``: dicts with ``lp`` (an object with m, n
    and the CSR/vector arrays), ``K``, ``eta``, ``omega`` and optionally ``gx``, ``gy``,
    ``checkpoint_every``.  Returns, per item, (status, x, y, grads or None)."""
    lib = load_library()
    mh = _Marshal(device)
    probs = (UnrolledProblem * max(1, len(items)))()
    outs = []
    for k, it in enumerate(items):
        inst = it["lp"]
        arrs = [inst.row_ptr, inst.col_idx, inst.val, inst.c, inst.lc, inst.uc, inst.lv, inst.uv]
        if device:
            import torch

            arrs = [a if _is_cuda_tensor(a) else torch.as_tensor(np.asarray(a)).cuda() for a in arrs]
        A, vecs = _lp_args(mh, inst.m, inst.n, *arrs)
        pr = probs[k]
        pr.m, pr.n, pr.A = inst.m, inst.n, A
        pr.c, pr.lc, pr.uc, pr.lv, pr.uv = vecs
        pr.K, pr.eta, pr.omega = int(it["K"]), float(it["eta"]), float(it.get("omega", 1.0))
        pr.checkpoint_every = int(it.get("checkpoint_every", 50))
        x, pr.x_out = mh.out(inst.n)
        y, pr.y_out = mh.out(inst.m)
        grads = None
        if it.get("gx") is not None:
            pr.gx, pr.gy = mh(it["gx"], "f64"), mh(it["gy"], "f64")
            grads = {}
            for key, ln in zip(GRAD_KEYS, (inst.n, inst.m, inst.m, inst.n, inst.n)):
                t, p_ = mh.out(ln)
                grads[key] = t
                setattr(pr, "grad_" + key, p_)
        outs.append((x, y, grads))
    prm = _params_for(device, params)
    status = (ctypes.c_int * max(1, len(items)))()
    if persistent:
        _check(lib.pdlp_unrolled_pdhg_batch_persistent(len(items), ctypes.addressof(probs),
                                                       ctypes.byref(prm), ctypes.addressof(status)))
    else:
        _check(lib.pdlp_unrolled_pdhg_batch(len(items), ctypes.addressof(probs), ctypes.byref(prm),
                                            int(concurrency), ctypes.addressof(status)))
    return [(status[k], *outs[k]) for k in range(len(items))]


def precondition(m, n, row_ptr, col_idx, val, **params):
    """pdlp_precondition: returns (d1, d2, scaled values) of Sec. 3's preconditioner."""
    lib = load_library()
    on_device = _is_cuda_tensor(val)
    mh = _Marshal(on_device)
    A = Csr()
    A.nnz = int(val.numel()) if on_device else int(len(val))
    A.row_ptr, A.col_idx, A.val = mh(row_ptr, "i64"), mh(col_idx, "i32"), mh(val, "f64")
    prm = _params_for(on_device, params)
    d1, p1 = mh.out(m)
    d2, p2 = mh.out(n)
    sv, p3 = mh.out(A.nnz)
    _check(lib.pdlp_precondition(m, n, ctypes.byref(A), ctypes.byref(prm), p1, p2, p3))
    return d1, d2, sv


def normalized_gap(m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv, x, y, x_ref, y_ref, omega,
                   **params) -> float:
    """pdlp_normalized_gap: mu(z, z_ref) of Sec. 3 for the LP as given."""
    lib = load_library()
    on_device = _is_cuda_tensor(val)
    mh = _Marshal(on_device)
    A, vecs = _lp_args(mh, m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv)
    pts = [mh(x, "f64"), mh(y, "f64"), mh(x_ref, "f64"), mh(y_ref, "f64")]
    prm = _params_for(on_device, params)
    mu = ctypes.c_double(math.nan)
    _check(lib.pdlp_normalized_gap(m, n, ctypes.byref(A), *vecs, *pts, float(omega),
                                   ctypes.byref(prm), ctypes.byref(mu)))
    return mu.value


KKT_FIELDS = ["rel_kkt", "rel_primal", "rel_dual", "rel_gap", "primal_res_l2", "dual_res_l2",
              "primal_res_inf", "dual_res_inf", "pobj", "dobj", "paper_gap"]


def kkt(m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv, x, y, **params) -> dict:
    """pdlp_kkt: residuals, objectives and gaps of (x, y) for the LP as given."""
    lib = load_library()
    on_device = _is_cuda_tensor(val)
    mh = _Marshal(on_device)
    A, vecs = _lp_args(mh, m, n, row_ptr, col_idx, val, c, lc, uc, lv, uv)
    pts = [mh(x, "f64"), mh(y, "f64")]
    prm = _params_for(on_device, params)
    out = np.zeros(len(KKT_FIELDS))
    _check(lib.pdlp_kkt(m, n, ctypes.byref(A), *vecs, *pts, ctypes.byref(prm), out.ctypes.data))
    return dict(zip(KKT_FIELDS, out.tolist()))


def kkt_products_noalloc(m, n, c, lc, uc, lv, uv, x, y, ax, aty, cuda_stream=None) -> dict:
    """pdlp_kkt_products_noalloc: the measures of ``kkt`` for a point whose products
    ax = A x and aty = A'y are given, without any allocation by the library.  Every
    array must be a float64 CUDA tensor on the current device."""
    import torch

    lib = load_library()
    args = [c, lc, uc, lv, uv, x, y, ax, aty]
    for t in args:
        if not (_is_cuda_tensor(t) and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("every array must be a contiguous float64 CUDA tensor")
    stream = cuda_stream if cuda_stream is not None else torch.cuda.current_stream().cuda_stream
    out = np.zeros(len(KKT_FIELDS))
    _check(lib.pdlp_kkt_products_noalloc(m, n, *[t.data_ptr() if t.numel() else None for t in args],
                                         stream, out.ctypes.data))
    return dict(zip(KKT_FIELDS, out.tolist()))


GATHER_METHODS = {"lsu": 0, "tma": 1, "hybrid": 2}


def gather_bench(method="lsu", elem_bytes=8, table_len=2_000_000, row_len=24,
                 nnz=50_000_000, degree_s=0.0, dmin=2.0, dmax=5000.0, reps=10) -> dict:
    """pdlp_gather_bench: the random-gather ceiling of the current GPU for the access
    pattern of the sparse products (a measurement; the data live on the device).
    degree_s <= 0: uniform indices; > 1: columns of a matrix with power-law degrees on
    [dmin, dmax], numbered by decreasing degree."""
    lib = load_library()
    out = np.zeros(4)
    _check(lib.pdlp_gather_bench(GATHER_METHODS[method], elem_bytes, int(table_len), row_len,
                                 int(nnz), float(degree_s), float(dmin), float(dmax), reps,
                                 out.ctypes.data))
    return dict(us=out[0], entries_per_s=out[1], max_diff_vs_lsu=out[2], entries=int(out[3]))

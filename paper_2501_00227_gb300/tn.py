"""Python binding of libtn (include/tn.h): argument marshalling only.

Every function named ``tn_*`` here calls the C entry point of the same name.
All arithmetic of a contraction runs in libtn's CUDA kernels; this module
only converts NumPy / PyTorch objects into pointers and sizes.  PyTorch is
used for device memory (workspaces) and streams.

If ``_build/libtn.so`` is missing the first call raises ``TNError``: there is
no fallback path.  Run ``paper_2501_00227_gb300.build.build()`` (or
``__graft_entry__.build()``) first.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

TN_OK, TN_EINVAL, TN_ENOMEM, TN_EOVERFLOW, TN_ETIMEOUT, TN_EAGAIN, TN_ECUDA = 0, -1, -2, -3, -4, -5, -6
TN_TROPICAL_F32, TN_TROPICAL_I32, TN_COUNTING_TROPICAL, TN_COUNT_MODP = 1, 2, 3, 4
TN_SIZE_MAX_K, TN_COUNTING_MAX_K = 5, 6
TN_KBEST_MAX = 4
KBEST = {"size_max": TN_SIZE_MAX_K, "counting_max": TN_COUNTING_MAX_K}
TN_I32_NEG_INF = -(1 << 30)
TN_MAX_PRIMES = 16
TN_RAW_BYTES = 128
TN_POLY_MAX_PRIMES = 32
TN_POLY_LIMBS = 32
TN_PROBLEM_INDEPENDENT_SET, TN_PROBLEM_SPIN_GLASS = 0, 1
PROBLEMS = {"is": TN_PROBLEM_INDEPENDENT_SET, "spin": TN_PROBLEM_SPIN_GLASS}

SEMIRINGS = {"tropical_f32": TN_TROPICAL_F32, "tropical_i32": TN_TROPICAL_I32,
             "counting": TN_COUNTING_TROPICAL, "modp": TN_COUNT_MODP}

#: the eight largest primes below 2^31
PRIMES31 = (2147483647, 2147483629, 2147483587, 2147483579,
            2147483563, 2147483549, 2147483543, 2147483497)


class tn_treesa_params_t(ctypes.Structure):
    _fields_ = [("sc_target", ctypes.c_double), ("beta_start", ctypes.c_double), ("beta_step", ctypes.c_double),
                ("beta_stop", ctypes.c_double), ("niters", ctypes.c_int32), ("ntrials", ctypes.c_int32),
                ("sc_weight", ctypes.c_double), ("rw_weight", ctypes.c_double), ("random_init", ctypes.c_int32),
                ("nthreads", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class tn_plan_info_t(ctypes.Structure):
    _fields_ = [("log2_tc", ctypes.c_double), ("log2_sc", ctypes.c_double), ("log2_rwc", ctypes.c_double),
                ("tc", ctypes.c_uint64), ("sc_elems", ctypes.c_uint64), ("rwc", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64 * 4), ("nsteps", ctypes.c_int32),
                ("nlaunch_steps", ctypes.c_int32), ("exec_table_bytes", ctypes.c_uint64),
                ("exec_tasks", ctypes.c_int32), ("exec_levels", ctypes.c_int32),
                ("exec_grid", ctypes.c_int32), ("exec_smem", ctypes.c_int32)]


class tn_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("max_i32", ctypes.c_int32), ("max_f32", ctypes.c_float),
                ("count", ctypes.c_uint64), ("nprimes", ctypes.c_int32),
                ("primes", ctypes.c_uint32 * TN_MAX_PRIMES), ("residues", ctypes.c_uint32 * TN_MAX_PRIMES),
                ("crt_nlimbs", ctypes.c_int32), ("crt_limbs", ctypes.c_uint32 * 32)]


class TNError(RuntimeError):
    def __init__(self, code, what="", detail=None):
        """detail: the message, when the library cannot describe the code
        (it is not loaded); otherwise tn_strerror's text is used."""
        self.code = code
        if detail is not None:
            msg = f"{what}: {detail} ({code})"
        else:
            msg = f"{what}: {tn_strerror(code)} ({code})" if what else f"{code}"
        super().__init__(msg)


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libtn.so (built in-tree); raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            # no tn_strerror here: it would call lib() under the held lock
            raise TNError(TN_EINVAL, "libtn.so", f"not built at {path}; run paper_2501_00227_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i32, u32, u64, i32p, u32p = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32))
        L.tn_plan.argtypes = [i32, i32p, i32, i32p, i32, ctypes.POINTER(vp)]
        L.tn_order_greedy.argtypes = [i32, i32p, i32, ctypes.c_double, i32, u64, i32p]
        L.tn_plan_info.argtypes = [vp, ctypes.c_int, i32, ctypes.POINTER(tn_plan_info_t)]
        L.tn_contract.argtypes = [vp, ctypes.c_int, u32p, i32, vp, ctypes.c_size_t, vp, ctypes.POINTER(tn_result_t)]
        L.tn_contract_async.argtypes = [vp, ctypes.c_int, u32p, i32, vp, ctypes.c_size_t, vp, vp]
        L.tn_contract_timed.argtypes = [vp, ctypes.c_int, u32p, i32, vp, ctypes.c_size_t, vp,
                                        ctypes.POINTER(tn_result_t), ctypes.POINTER(ctypes.c_float),
                                        i32p, ctypes.POINTER(ctypes.c_uint64)]
        L.tn_contract_trace.argtypes = [vp, ctypes.c_int, u32p, i32, vp, ctypes.c_size_t, vp, vp, i32p, i32p,
                                        i32p, ctypes.POINTER(tn_result_t)]
        L.tn_contract_static.argtypes = [vp, ctypes.c_int, u32p, i32, vp, ctypes.POINTER(tn_result_t)]
        L.tn_tune_set.argtypes = [i32p, i32]
        L.tn_kbest_workspace_bytes.argtypes = [vp, ctypes.c_int, i32, ctypes.POINTER(u64)]
        L.tn_contract_kbest.argtypes = [vp, ctypes.c_int, i32, vp, ctypes.c_size_t, vp, i32p,
                                        ctypes.POINTER(u64), i32p]
        L.tn_modp_gemm_limb.argtypes = [u32p, i32, vp, vp, vp, i32, i32, i32, i32, vp]
        L.tn_modp_gemm_umma.argtypes = [u32p, i32, vp, vp, vp, i32, i32, i32, i32, vp]
        L.tn_plan_step_info.argtypes = [vp, ctypes.c_int, i32, i32p, i32]
        L.tn_contract_modp_x.argtypes = [vp, u32p, u32p, i32, vp, ctypes.c_size_t, vp, u32p]
        L.tn_independence_polynomial.argtypes = [vp, u32p, i32, i32, vp, ctypes.c_size_t, vp, u32p, u32p, i32p]
        L.tn_weighted_workspace_bytes.argtypes = [vp, ctypes.c_int, i32, ctypes.POINTER(u64)]
        L.tn_single_config_workspace_bytes.argtypes = [vp, ctypes.POINTER(u64)]
        L.tn_order_treesa.argtypes = [i32, i32p, i32, ctypes.POINTER(tn_treesa_params_t), i32p,
                                      ctypes.POINTER(ctypes.c_double)]
        L.tn_order_treesa_sliced.argtypes = [i32, i32p, i32, ctypes.POINTER(tn_treesa_params_t), i32, i32p, i32,
                                             i32p, i32p, ctypes.POINTER(ctypes.c_double)]
        L.tn_set_wait_timeout_ns.argtypes = [u64]
        L.tn_slice_labels.argtypes = [i32, i32p, i32, i32p, i32, i32, i32p, ctypes.POINTER(ctypes.c_double)]
        L.tn_plan_sliced.argtypes = [i32, i32p, i32, i32p, i32, i32p, i32, ctypes.POINTER(vp)]
        L.tn_contract_sliced.argtypes = [vp, ctypes.c_int, i32, i32p, i32p, u32p, u32p, i32, u64, u64, vp,
                                         ctypes.c_size_t, vp, ctypes.POINTER(tn_result_t)]
        L.tn_result_combine.argtypes = [ctypes.c_int, ctypes.POINTER(tn_result_t), ctypes.POINTER(tn_result_t),
                                        ctypes.POINTER(tn_result_t)]
        L.tn_sliced_workspace_bytes.argtypes = [vp, ctypes.c_int, i32, i32, ctypes.POINTER(u64)]
        L.tn_single_config_max.argtypes = [vp, i32, i32p, i32p, vp, ctypes.c_size_t, vp, i32p,
                                           ctypes.POINTER(ctypes.c_uint8)]
        L.tn_contract_weighted.argtypes = [vp, ctypes.c_int, i32, i32p, i32p, u32p, u32p, i32, vp, ctypes.c_size_t,
                                           vp, ctypes.POINTER(tn_result_t)]
        L.tn_weighted_polynomial.argtypes = [vp, i32, i32p, i32p, u32p, i32, i32, vp, ctypes.c_size_t, vp, u32p,
                                             u32p, i32p]
        L.tn_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_int, u32p, i32, ctypes.POINTER(vp)]
        L.tn_batch_info.argtypes = [vp, ctypes.POINTER(u64), i32p, i32p, ctypes.POINTER(u64)]
        L.tn_batch_contract.argtypes = [vp, vp, ctypes.c_size_t, vp, vp]
        L.tn_batch_contract_graph.argtypes = [vp, vp, ctypes.c_size_t, vp, vp]
        L.tn_batch_destroy.argtypes = [vp]
        L.tn_result_decode.argtypes = [ctypes.c_int, u32p, i32, vp, ctypes.POINTER(tn_result_t)]
        L.tn_contract_pair.argtypes = [ctypes.c_int, u32p, i32, vp, i32p, i32, vp, i32p, i32, i32p, i32, vp, vp]
        L.tn_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
        L.tn_submit.argtypes = [vp, vp, ctypes.c_int, u32p, i32, ctypes.POINTER(u64)]
        L.tn_poll.argtypes = [vp, u64, ctypes.POINTER(tn_result_t)]
        L.tn_server_completed.argtypes = [vp, ctypes.POINTER(u64), i32, i32p]
        L.tn_alu_peak.argtypes = [i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.tn_plan_destroy.argtypes = [vp]
        L.tn_server_destroy.argtypes = [vp]
        L.tn_strerror.argtypes = [ctypes.c_int]
        L.tn_strerror.restype = ctypes.c_char_p
        _lib = L
        return L


def declared_symbols() -> list[str]:
    """Names of every function include/tn.h declares."""
    hdr = os.path.join(_build.INCLUDE, "tn.h")
    with open(hdr) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_]+)\s*\(", text)))


# --------------------------------------------------------------------- helpers

def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _primes(primes):
    if primes is None:
        return None, 0
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    return pr, int(pr.size)


def _u32p(pr):
    return None if pr is None else pr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _check(rc, what):
    if rc != TN_OK:
        raise TNError(rc, what)


def _sr(semiring):
    return SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)


def result_dict(r: tn_result_t, semiring) -> dict:
    s = _sr(semiring)
    out = {"status": int(r.status)}
    if s in (TN_TROPICAL_F32, TN_TROPICAL_I32, TN_COUNTING_TROPICAL):
        out["max"] = None if r.max_i32 == -(2 ** 31) else int(r.max_i32)
        out["max_f32"] = float(r.max_f32)
    if s == TN_COUNTING_TROPICAL:
        out["count"] = int(r.count)
    if s == TN_COUNT_MODP:
        k = int(r.nprimes)
        out["primes"] = [int(x) for x in r.primes[:k]]
        out["residues"] = [int(x) for x in r.residues[:k]]
        x = 0
        for i in range(int(r.crt_nlimbs)):
            x |= int(r.crt_limbs[i]) << (32 * i)
        M = 1
        for p in out["primes"]:
            M *= p
        out["crt"], out["modulus"] = x, M
    return out


# --------------------------------------------------------------------- C ABI

def tn_strerror(code: int) -> str:
    return lib().tn_strerror(int(code)).decode()


def tn_order_greedy(n, edges, alpha: float = 0.0, nrepeat: int = 10, seed: int = 0) -> np.ndarray:
    e = _i32(edges).reshape(-1, 2)
    m = e.shape[0]
    out = np.zeros((max(n + m - 1, 0), 2), dtype=np.int32)
    _check(lib().tn_order_greedy(int(n), _p32(e), m, float(alpha), int(nrepeat), int(seed) & (2 ** 64 - 1),
                                 _p32(out)), "tn_order_greedy")
    return out


def tn_plan(n, edges, order) -> int:
    e = _i32(edges).reshape(-1, 2)
    o = _i32(order).reshape(-1, 2)
    h = ctypes.c_void_p()
    _check(lib().tn_plan(int(n), _p32(e), e.shape[0], _p32(o), o.shape[0], ctypes.byref(h)), "tn_plan")
    return h.value


def tn_plan_info(plan, semiring=TN_TROPICAL_I32, nprimes: int = 1) -> dict:
    info = tn_plan_info_t()
    _check(lib().tn_plan_info(plan, _sr(semiring), int(nprimes), ctypes.byref(info)), "tn_plan_info")
    return {"log2_tc": info.log2_tc, "log2_sc": info.log2_sc, "log2_rwc": info.log2_rwc,
            "tc": int(info.tc), "sc": int(info.sc_elems), "rwc": int(info.rwc),
            "peak_bytes": [int(x) for x in info.peak_bytes], "nsteps": int(info.nsteps),
            "nlaunch_steps": int(info.nlaunch_steps), "exec_table_bytes": int(info.exec_table_bytes),
            "exec_tasks": int(info.exec_tasks), "exec_levels": int(info.exec_levels),
            "exec_grid": int(info.exec_grid), "exec_smem": int(info.exec_smem)}


def tn_plan_destroy(plan):
    if plan:
        lib().tn_plan_destroy(plan)


def tn_contract(plan, semiring, primes, ws_ptr: int, ws_bytes: int, stream: int) -> dict:
    pr, k = _primes(primes)
    r = tn_result_t()
    _check(lib().tn_contract(plan, _sr(semiring), _u32p(pr), k, ctypes.c_void_p(ws_ptr), ws_bytes,
                             ctypes.c_void_p(stream), ctypes.byref(r)), "tn_contract")
    return result_dict(r, semiring)


def tn_contract_timed(plan, semiring, primes, ws_ptr: int, ws_bytes: int, stream: int, nsteps: int):
    """(result dict, per-step ms, per-step kernel id, per-step ops)."""
    pr, k = _primes(primes)
    r = tn_result_t()
    ms = np.zeros(nsteps, dtype=np.float32)
    kern = np.zeros(nsteps, dtype=np.int32)
    ops = np.zeros(nsteps, dtype=np.uint64)
    _check(lib().tn_contract_timed(plan, _sr(semiring), _u32p(pr), k, ctypes.c_void_p(ws_ptr), ws_bytes,
                                   ctypes.c_void_p(stream), ctypes.byref(r),
                                   ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _p32(kern),
                                   ops.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "tn_contract_timed")
    return result_dict(r, semiring), ms, kern, ops


def tn_contract_trace(plan, semiring, primes, ws_ptr: int, ws_bytes: int, stream: int, trace_ptr: int,
                      ntasks: int, nsteps: int):
    """(result dict, task_step, task_kind, step_level); the trace itself is in
    the caller's device buffer at trace_ptr (8 uint64 per task)."""
    pr, k = _primes(primes)
    r = tn_result_t()
    ts = np.zeros(ntasks, dtype=np.int32)
    tk = np.zeros(ntasks, dtype=np.int32)
    lv = np.zeros(nsteps, dtype=np.int32)
    _check(lib().tn_contract_trace(plan, _sr(semiring), _u32p(pr), k, ctypes.c_void_p(ws_ptr), ws_bytes,
                                   ctypes.c_void_p(stream), ctypes.c_void_p(trace_ptr), _p32(ts), _p32(tk),
                                   _p32(lv), ctypes.byref(r)), "tn_contract_trace")
    return result_dict(r, semiring), ts, tk, lv


def _kb(kind):
    return KBEST[kind] if isinstance(kind, str) else int(kind)


def tn_kbest_workspace_bytes(plan, kind, k: int) -> int:
    """Workspace bytes of tn_contract_kbest (kind 'size_max' or 'counting_max')."""
    out = ctypes.c_uint64()
    _check(lib().tn_kbest_workspace_bytes(plan, _kb(kind), int(k), ctypes.byref(out)), "tn_kbest_workspace_bytes")
    return int(out.value)


def tn_contract_kbest(plan, kind, k: int, ws_ptr: int, ws_bytes: int, stream: int) -> dict:
    """SizeMax(k) / CountingMax(k) in one contraction (Sec. 5.3, Table 1).
    'size_max': {"values": the k largest set sizes (None for -inf)};
    'counting_max': {"max": alpha, "counts": [c_alpha, c_(alpha-1), ...]};
    both with "status"."""
    vals = np.zeros(max(int(k), 1), dtype=np.int32)
    cnts = np.zeros(max(int(k), 1), dtype=np.uint64)
    status = ctypes.c_int32()
    _check(lib().tn_contract_kbest(plan, _kb(kind), int(k), ctypes.c_void_p(ws_ptr), ws_bytes,
                                   ctypes.c_void_p(stream), _p32(vals),
                                   cnts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(status)),
           "tn_contract_kbest")
    if _kb(kind) == TN_SIZE_MAX_K:
        return {"status": int(status.value), "values": [None if v == -2**31 else int(v) for v in vals[:k]]}
    d = int(vals[0])
    return {"status": int(status.value), "max": None if d == -2**31 else d, "counts": [int(c) for c in cnts[:k]]}


TN_STATIC_WORKSPACE_BYTES = 64 * 1024 * 1024


def tn_contract_static(plan, semiring, primes, stream: int) -> dict:
    """Contraction whose workspace is the library's static device array (no
    device allocation; for callers that cannot call cudaMalloc)."""
    pr, k = _primes(primes)
    r = tn_result_t()
    _check(lib().tn_contract_static(plan, _sr(semiring), _u32p(pr), k, ctypes.c_void_p(stream), ctypes.byref(r)),
           "tn_contract_static")
    return result_dict(r, semiring)


def tn_contract_async(plan, semiring, primes, ws_ptr: int, ws_bytes: int, stream: int, raw_ptr: int):
    pr, k = _primes(primes)
    _check(lib().tn_contract_async(plan, _sr(semiring), _u32p(pr), k, ctypes.c_void_p(ws_ptr), ws_bytes,
                                   ctypes.c_void_p(stream), ctypes.c_void_p(raw_ptr)), "tn_contract_async")


def tn_result_decode(semiring, primes, raw: bytes) -> dict:
    pr, k = _primes(primes)
    buf = ctypes.create_string_buffer(bytes(raw), TN_RAW_BYTES)
    r = tn_result_t()
    _check(lib().tn_result_decode(_sr(semiring), _u32p(pr), k, ctypes.cast(buf, ctypes.c_void_p),
                                  ctypes.byref(r)), "tn_result_decode")
    return result_dict(r, semiring)


def tn_contract_modp_x(plan, primes, xs, ws_ptr: int, ws_bytes: int, stream: int) -> list:
    """Residues I(G, xs[q]) mod primes[q] of the independence polynomial, one
    slot per (prime, point) pair (at most TN_MAX_PRIMES slots)."""
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32).reshape(-1))
    xv = np.ascontiguousarray(np.asarray(xs, dtype=np.uint32).reshape(-1))
    if pr.size != xv.size:
        raise TNError(TN_EINVAL, "tn_contract_modp_x: primes and xs differ in length")
    out = np.zeros(pr.size, dtype=np.uint32)
    _check(lib().tn_contract_modp_x(plan, _u32p(pr), _u32p(xv), pr.size, ctypes.c_void_p(ws_ptr), ws_bytes,
                                    ctypes.c_void_p(stream), _u32p(out)), "tn_contract_modp_x")
    return [int(v) for v in out]


def tn_independence_polynomial(plan, primes, degree: int, ws_ptr: int, ws_bytes: int, stream: int):
    """Coefficients c_0 .. c_degree of the independence polynomial (exact
    when prod(primes) exceeds every coefficient) and their residues,
    shape (degree + 1, len(primes))."""
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32).reshape(-1))
    d = int(degree)
    res = np.zeros((max(d + 1, 1), max(pr.size, 1)), dtype=np.uint32)
    limbs = np.zeros((max(d + 1, 1), TN_POLY_LIMBS), dtype=np.uint32)
    nl = np.zeros(max(d + 1, 1), dtype=np.int32)
    _check(lib().tn_independence_polynomial(plan, _u32p(pr), pr.size, d, ctypes.c_void_p(ws_ptr), ws_bytes,
                                            ctypes.c_void_p(stream), _u32p(res), _u32p(limbs), _p32(nl)),
           "tn_independence_polynomial")
    coeffs = [sum(int(limbs[k, i]) << (32 * i) for i in range(int(nl[k]))) for k in range(d + 1)]
    return coeffs, res


def _opt_i32(w):
    """int32 array of weights (or None) and its pointer (or NULL)."""
    if w is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(w, dtype=np.int32).reshape(-1))
    return a, _p32(a)


def _problem(problem) -> int:
    return PROBLEMS[problem] if isinstance(problem, str) else int(problem)


def tn_weighted_workspace_bytes(plan, semiring, nslots: int = 1) -> int:
    out = ctypes.c_uint64()
    _check(lib().tn_weighted_workspace_bytes(plan, _sr(semiring), int(nslots), ctypes.byref(out)),
           "tn_weighted_workspace_bytes")
    return int(out.value)


def tn_contract_weighted(plan, semiring, problem, edge_w, vertex_w, primes, xs, ws_ptr: int, ws_bytes: int,
                         stream: int) -> dict:
    """Weighted IS / spin-glass contraction; for "modp" one residue per slot
    (primes[q], xs[q]) in result["residues"]."""
    ew, ewp = _opt_i32(edge_w)
    vw, vwp = _opt_i32(vertex_w)
    if _sr(semiring) == TN_COUNT_MODP:
        pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32).reshape(-1))
        xv = np.ascontiguousarray(np.asarray(xs, dtype=np.uint32).reshape(-1))
        if pr.size != xv.size:
            raise TNError(TN_EINVAL, "tn_contract_weighted: primes and xs differ in length")
        prp, xvp, k = _u32p(pr), _u32p(xv), pr.size
    else:
        prp, xvp, k = None, None, 0
    r = tn_result_t()
    _check(lib().tn_contract_weighted(plan, _sr(semiring), _problem(problem), ewp, vwp, prp, xvp, k,
                                      ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream), ctypes.byref(r)),
           "tn_contract_weighted")
    out = {"status": int(r.status)}
    if _sr(semiring) == TN_COUNT_MODP:
        out["primes"] = [int(x) for x in r.primes[:k]]
        out["residues"] = [int(x) for x in r.residues[:k]]
    else:
        out["max"] = None if r.max_i32 == -(2 ** 31) else int(r.max_i32)
        if _sr(semiring) == TN_COUNTING_TROPICAL:
            out["count"] = int(r.count)
    return out


def tn_weighted_polynomial(plan, problem, edge_w, vertex_w, primes, degree: int, ws_ptr: int, ws_bytes: int,
                           stream: int):
    """Coefficients of a weighted network's generating polynomial and their
    residues (see include/tn.h)."""
    ew, ewp = _opt_i32(edge_w)
    vw, vwp = _opt_i32(vertex_w)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32).reshape(-1))
    d = int(degree)
    res = np.zeros((max(d + 1, 1), max(pr.size, 1)), dtype=np.uint32)
    limbs = np.zeros((max(d + 1, 1), TN_POLY_LIMBS), dtype=np.uint32)
    nl = np.zeros(max(d + 1, 1), dtype=np.int32)
    _check(lib().tn_weighted_polynomial(plan, _problem(problem), ewp, vwp, _u32p(pr), pr.size, d,
                                        ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream), _u32p(res),
                                        _u32p(limbs), _p32(nl)), "tn_weighted_polynomial")
    coeffs = [sum(int(limbs[k, i]) << (32 * i) for i in range(int(nl[k]))) for k in range(d + 1)]
    return coeffs, res


def tn_order_treesa(n, edges, *, sc_target: float = 20.0, betas=(1.0, 0.05, 15.0), niters: int = 50,
                    ntrials: int = 10, sc_weight: float = 1.0, rw_weight: float = 0.2, random_init: bool = False,
                    nthreads: int = 0, seed: int = 0):
    """TreeSA order (Sec. 4.2.2) and log2 (tc, sc, rwc) of it.  The defaults
    are the paper's except the first inverse temperature (1.0, not 0.01): on
    this cost's log2 scale a start hotter than about 0.3 melts the greedy
    starting trees of 100+ vertex graphs beyond what the schedule recovers."""
    e = _i32(edges).reshape(-1, 2)
    prm = _treesa_params(sc_target, betas, niters, ntrials, sc_weight, rw_weight, random_init, nthreads, seed)
    order = np.zeros((max(int(n) + len(e) - 1, 0), 2), dtype=np.int32)
    lg = (ctypes.c_double * 3)()
    _check(lib().tn_order_treesa(int(n), _p32(e), len(e), ctypes.byref(prm), _p32(order), lg), "tn_order_treesa")
    return order, tuple(float(x) for x in lg)


def _treesa_params(sc_target, betas, niters, ntrials, sc_weight, rw_weight, random_init, nthreads, seed):
    return tn_treesa_params_t(float(sc_target), float(betas[0]), float(betas[1]), float(betas[2]), int(niters),
                              int(ntrials), float(sc_weight), float(rw_weight), int(bool(random_init)),
                              int(nthreads), int(seed))


def tn_order_treesa_sliced(n, edges, *, nslices: int = 0, fixed_slices=(), sc_target: float = 20.0,
                           betas=(1.0, 0.05, 15.0), niters: int = 50, ntrials: int = 10, sc_weight: float = 1.0,
                           rw_weight: float = 0.2, random_init: bool = False, nthreads: int = 0, seed: int = 0):
    """TreeSA with slicing (Sec. 4.2.2): `fixed_slices` sliced from the
    start, `nslices` more picked while annealing.  Returns (order, sliced
    labels -- the fixed ones first --, log2 (work of all slices, largest
    intermediate of one slice, reads and writes of all slices))."""
    e = _i32(edges).reshape(-1, 2)
    fx = _i32(list(fixed_slices)).reshape(-1)
    prm = _treesa_params(sc_target, betas, niters, ntrials, sc_weight, rw_weight, random_init, nthreads, seed)
    order = np.zeros((max(int(n) + len(e) - 1, 0), 2), dtype=np.int32)
    sl = np.zeros(max(fx.size + int(nslices), 1), dtype=np.int32)
    lg = (ctypes.c_double * 3)()
    _check(lib().tn_order_treesa_sliced(int(n), _p32(e), len(e), ctypes.byref(prm), int(nslices),
                                        _p32(fx) if fx.size else None, fx.size, _p32(order), _p32(sl), lg),
           "tn_order_treesa_sliced")
    return order, sl[: fx.size + int(nslices)], tuple(float(x) for x in lg)


def tn_set_wait_timeout_ns(ns: int):
    """Limit of the executor's dependency waits for the launches that follow
    (0: the default, 2 s)."""
    _check(lib().tn_set_wait_timeout_ns(int(ns)), "tn_set_wait_timeout_ns")


def tn_slice_labels(n, edges, order, nslices: int):
    """Labels to slice for `order` and log2 (work of all slices, largest
    intermediate of one slice)."""
    e = _i32(edges).reshape(-1, 2)
    o = _i32(order).reshape(-1, 2)
    out = np.zeros(max(int(nslices), 1), dtype=np.int32)
    lg = (ctypes.c_double * 2)()
    _check(lib().tn_slice_labels(int(n), _p32(e), len(e), _p32(o), len(o), int(nslices), _p32(out), lg),
           "tn_slice_labels")
    return out[: int(nslices)], (float(lg[0]), float(lg[1]))


def tn_plan_sliced(n, edges, order, sliced):
    e = _i32(edges).reshape(-1, 2)
    o = _i32(order).reshape(-1, 2)
    sl = _i32(sliced).reshape(-1)
    out = ctypes.c_void_p()
    _check(lib().tn_plan_sliced(int(n), _p32(e), len(e), _p32(o), len(o), _p32(sl), sl.size, ctypes.byref(out)),
           "tn_plan_sliced")
    return out.value


def _result_from(d, semiring) -> "tn_result_t":
    r = tn_result_t()
    r.status = d.get("status", 0)
    if _sr(semiring) == TN_COUNT_MODP:
        r.nprimes = len(d["primes"])
        for q, (p, x) in enumerate(zip(d["primes"], d["residues"])):
            r.primes[q], r.residues[q] = p, x
    else:
        mx = d.get("max")
        r.max_i32 = -(2 ** 31) if mx is None else int(mx)
        r.max_f32 = float("-inf") if mx is None else float(mx)
        r.count = int(d.get("count", 0))
    return r


def _result_dict(r, semiring) -> dict:
    out = {"status": int(r.status)}
    if _sr(semiring) == TN_COUNT_MODP:
        out["primes"] = [int(x) for x in r.primes[: r.nprimes]]
        out["residues"] = [int(x) for x in r.residues[: r.nprimes]]
    else:
        out["max"] = None if r.max_i32 == -(2 ** 31) else int(r.max_i32)
        if _sr(semiring) == TN_COUNTING_TROPICAL:
            out["count"] = int(r.count)
    return out


def tn_sliced_workspace_bytes(plan, semiring, nslots: int = 1, batch: int = 1) -> int:
    out = ctypes.c_uint64()
    _check(lib().tn_sliced_workspace_bytes(plan, _sr(semiring), int(nslots), int(batch), ctypes.byref(out)),
           "tn_sliced_workspace_bytes")
    return int(out.value)


def tn_result_combine(semiring, a: dict, b: dict) -> dict:
    """a (+) b in the element type (results as returned by the contract calls)."""
    ra, rb, rc = _result_from(a, semiring), _result_from(b, semiring), tn_result_t()
    _check(lib().tn_result_combine(_sr(semiring), ctypes.byref(ra), ctypes.byref(rb), ctypes.byref(rc)),
           "tn_result_combine")
    return _result_dict(rc, semiring)


def tn_contract_sliced(plan, semiring, problem, edge_w, vertex_w, primes, xs, slice_begin: int, slice_end: int,
                       ws_ptr: int, ws_bytes: int, stream: int) -> dict:
    ew, ewp = _opt_i32(edge_w)
    vw, vwp = _opt_i32(vertex_w)
    if _sr(semiring) == TN_COUNT_MODP:
        pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32).reshape(-1))
        xv = np.ascontiguousarray(np.asarray(xs, dtype=np.uint32).reshape(-1))
        prp, xvp, k = _u32p(pr), _u32p(xv), pr.size
    else:
        prp, xvp, k = None, None, 0
    r = tn_result_t()
    _check(lib().tn_contract_sliced(plan, _sr(semiring), _problem(problem), ewp, vwp, prp, xvp, k, int(slice_begin),
                                    int(slice_end), ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream),
                                    ctypes.byref(r)), "tn_contract_sliced")
    return _result_dict(r, semiring)


def tn_single_config_workspace_bytes(plan) -> int:
    out = ctypes.c_uint64()
    _check(lib().tn_single_config_workspace_bytes(plan, ctypes.byref(out)), "tn_single_config_workspace_bytes")
    return int(out.value)


def tn_single_config_max(plan, problem, edge_w, vertex_w, n: int, ws_ptr: int, ws_bytes: int, stream: int):
    """(maximum, configuration as a uint8 array of n 0/1 values)."""
    ew, ewp = _opt_i32(edge_w)
    vw, vwp = _opt_i32(vertex_w)
    val = np.zeros(1, dtype=np.int32)
    cfg = np.zeros(max(int(n), 1), dtype=np.uint8)
    _check(lib().tn_single_config_max(plan, _problem(problem), ewp, vwp, ctypes.c_void_p(ws_ptr), ws_bytes,
                                      ctypes.c_void_p(stream), _p32(val),
                                      cfg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "tn_single_config_max")
    return int(val[0]), cfg[: int(n)]


def _is_prime32(p: int) -> bool:
    """Deterministic Miller-Rabin for p < 2^32 (bases 2, 7, 61)."""
    if p < 2:
        return False
    for sp in (2, 3, 5, 7, 11, 13, 61):
        if p % sp == 0:
            return p == sp
    d, r = p - 1, 0
    while d % 2 == 0:
        d, r = d // 2, r + 1
    for a in (2, 7, 61):
        x = pow(a, d, p)
        if x in (1, p - 1):
            continue
        for _ in range(r - 1):
            x = x * x % p
            if x == p - 1:
                break
        else:
            return False
    return True


def primes31(count: int) -> tuple:
    """The `count` largest primes below 2^31 (the first eight are PRIMES31)."""
    out, p = [], (1 << 31) - 1
    while len(out) < count:
        if _is_prime32(p):
            out.append(p)
        p -= 1
    return tuple(out)


def tn_contract_pair(semiring, primes, a_ptr, la, b_ptr, lb, lc, c_ptr, stream: int):
    pr, k = _primes(primes)
    la, lb, lc = _i32(la).reshape(-1), _i32(lb).reshape(-1), _i32(lc).reshape(-1)
    _check(lib().tn_contract_pair(_sr(semiring), _u32p(pr), k, ctypes.c_void_p(a_ptr), _p32(la), la.size,
                                  ctypes.c_void_p(b_ptr), _p32(lb), lb.size, _p32(lc), lc.size,
                                  ctypes.c_void_p(c_ptr), ctypes.c_void_p(stream)), "tn_contract_pair")


def tn_modp_gemm_limb(primes, a_ptr: int, b_ptr: int, c_ptr: int, batch: int, m: int, n: int, k: int,
                      stream: int) -> None:
    """Tensor-core (8-bit limb) mod-p batched GEMM, an ablation of the
    CUDA-core path: C[q,b] = A[q,b] B[q,b]^T mod primes[q]."""
    pr, kk = _primes(primes)
    _check(lib().tn_modp_gemm_limb(_u32p(pr), kk, ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr),
                                   ctypes.c_void_p(c_ptr), int(batch), int(m), int(n), int(k),
                                   ctypes.c_void_p(stream)), "tn_modp_gemm_limb")


def tn_modp_gemm_umma(primes, a_ptr: int, b_ptr: int, c_ptr: int, batch: int, m: int, n: int, k: int,
                      stream: int) -> None:
    """The same product on tcgen05 tensor cores (bf16 limbs, fp32 tensor-memory
    accumulators); waits for the stream."""
    pr, kk = _primes(primes)
    _check(lib().tn_modp_gemm_umma(_u32p(pr), kk, ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr),
                                   ctypes.c_void_p(c_ptr), int(batch), int(m), int(n), int(k),
                                   ctypes.c_void_p(stream)), "tn_modp_gemm_umma")


def tn_tune_set(entries) -> None:
    """Install measured launch shapes: rows (semiring, nb, nm, nn, nk, tile,
    split); an empty list removes the table."""
    rows = [[int(SEMIRINGS[r[0]]) if isinstance(r[0], str) else int(r[0]), *map(int, r[1:])] for r in entries]
    arr = _i32(np.array(rows, dtype=np.int32).reshape(-1)) if rows else np.zeros(1, dtype=np.int32)
    _check(lib().tn_tune_set(_p32(arr), len(rows)), "tn_tune_set")


def tn_plan_step_info(plan, semiring, nprimes: int = 1) -> np.ndarray:
    """(nsteps, 10) int32: exec index, level, kernel, tile, split, tasks, nb,
    nm, nn, nk of every pairwise step (plan order)."""
    n = tn_plan_info(plan, semiring, nprimes)["nsteps"]
    out = np.zeros(10 * max(n, 1), dtype=np.int32)
    _check(lib().tn_plan_step_info(plan, _sr(semiring), int(nprimes), _p32(out), n), "tn_plan_step_info")
    return out[:10 * n].reshape(n, 10)


def tn_server_create(hbm_budget_bytes: int, max_inflight: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().tn_server_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(h)), "tn_server_create")
    return h.value


def tn_submit(server, plan, semiring, primes=None) -> int:
    pr, k = _primes(primes)
    t = ctypes.c_uint64()
    _check(lib().tn_submit(server, plan, _sr(semiring), _u32p(pr), k, ctypes.byref(t)), "tn_submit")
    return int(t.value)


def tn_poll(server, ticket: int, semiring):
    """Result dict once ready, None while TN_EAGAIN."""
    r = tn_result_t()
    rc = lib().tn_poll(server, int(ticket), ctypes.byref(r))
    if rc == TN_EAGAIN:
        return None
    _check(rc, "tn_poll")
    return result_dict(r, semiring)


def tn_server_completed(server, max_tickets: int = 4096) -> list:
    """Tickets finished since the last call (each reported once)."""
    buf = (ctypes.c_uint64 * max(int(max_tickets), 1))()
    n = ctypes.c_int32()
    _check(lib().tn_server_completed(server, buf, int(max_tickets), ctypes.byref(n)), "tn_server_completed")
    return [int(buf[i]) for i in range(n.value)]


def tn_alu_peak(kind: str, iters: int = 1 << 14, stream: int = 0) -> float:
    """Register-only Tops/s of the "maxplus", "modp" or "maxplus16x2" inner step."""
    out = ctypes.c_double()
    _check(lib().tn_alu_peak({"maxplus": 0, "modp": 1, "maxplus16x2": 2}[kind], int(iters), ctypes.c_void_p(stream),
                             ctypes.byref(out)), "tn_alu_peak")
    return float(out.value)


def tn_server_destroy(server):
    if server:
        lib().tn_server_destroy(server)


def tn_batch_create(plans, semiring, primes=None) -> int:
    handles = (ctypes.c_void_p * len(plans))(*[p.handle if hasattr(p, "handle") else p for p in plans])
    pr, k = _primes(primes)
    h = ctypes.c_void_p()
    _check(lib().tn_batch_create(handles, len(plans), _sr(semiring), _u32p(pr), k, ctypes.byref(h)),
           "tn_batch_create")
    return h.value


def tn_batch_info(batch) -> dict:
    ws, tb = ctypes.c_uint64(), ctypes.c_uint64()
    ta, lv = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().tn_batch_info(batch, ctypes.byref(ws), ctypes.byref(ta), ctypes.byref(lv), ctypes.byref(tb)),
           "tn_batch_info")
    return {"workspace_bytes": int(ws.value), "tasks": int(ta.value), "levels": int(lv.value),
            "table_bytes": int(tb.value)}


def tn_batch_contract(batch, ws_ptr: int, ws_bytes: int, stream: int, raw_ptr: int):
    _check(lib().tn_batch_contract(batch, ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream),
                                   ctypes.c_void_p(raw_ptr)), "tn_batch_contract")


def tn_batch_contract_graph(batch, ws_ptr: int, ws_bytes: int, stream: int, raw_ptr: int):
    _check(lib().tn_batch_contract_graph(batch, ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream),
                                         ctypes.c_void_p(raw_ptr)), "tn_batch_contract_graph")


def tn_batch_destroy(batch):
    if batch:
        lib().tn_batch_destroy(batch)


# --------------------------------------------------------------------- objects

class Plan:
    """A contraction plan (graph + order) owning its libtn handle."""

    def __init__(self, n, edges, order=None, *, nrepeat: int = 10, seed: int = 0, alpha: float = 0.0,
                 optimizer: str = "greedy", treesa=None, sliced=None):
        """order None: found by `optimizer` -- "greedy" (Sec. 4.2.1, nrepeat /
        seed / alpha) or "treesa" (Sec. 4.2.2, keyword arguments of
        tn_order_treesa in the dict `treesa`, seed defaulting to `seed`;
        with "nslices" or "fixed_slices" among them, the labels sliced while
        annealing, tn_order_treesa_sliced, become the plan's slices).
        sliced: vertex labels to slice (tn_plan_sliced; contract with
        contract_sliced), or an int s to pick s labels with tn_slice_labels."""
        self.n = int(n)
        self.edges = _i32(edges).reshape(-1, 2)
        if order is not None:
            self.order = _i32(order).reshape(-1, 2)
        elif optimizer == "treesa":
            kw = dict(treesa or {})
            kw.setdefault("seed", seed)
            if "nslices" in kw or "fixed_slices" in kw:
                if sliced is not None:
                    raise TNError(TN_EINVAL, "slices come from the annealing or from `sliced`, not both")
                self.order, sliced, _ = tn_order_treesa_sliced(n, self.edges, **kw)
            else:
                self.order, _ = tn_order_treesa(n, self.edges, **kw)
        elif optimizer == "greedy":
            self.order = tn_order_greedy(n, self.edges, alpha, nrepeat, seed)
        else:
            raise TNError(TN_EINVAL, f"unknown optimizer {optimizer!r}")
        if isinstance(sliced, (int, np.integer)):
            sliced = tn_slice_labels(self.n, self.edges, self.order, int(sliced))[0]
        self.sliced = None if sliced is None else _i32(sliced).reshape(-1)
        self.handle = (tn_plan(self.n, self.edges, self.order) if self.sliced is None
                       else tn_plan_sliced(self.n, self.edges, self.order, self.sliced))

    def info(self, semiring=TN_TROPICAL_I32, nprimes: int = 1) -> dict:
        return tn_plan_info(self.handle, semiring, nprimes)

    def workspace_bytes(self, semiring, nprimes: int = 1) -> int:
        return self.info(semiring, nprimes)["peak_bytes"][_sr(semiring) - 1]

    def contract(self, semiring, primes=None, workspace=None, stream=None) -> dict:
        """Contract on the current CUDA device; allocates a torch workspace if none is given."""
        import torch
        nprimes = 0 if primes is None else len(primes)
        need = self.workspace_bytes(semiring, max(nprimes, 1))
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_contract(self.handle, semiring, primes, workspace.data_ptr(), workspace.numel(),
                           st.cuda_stream)

    def kbest(self, kind, k: int, workspace=None, stream=None) -> dict:
        """SizeMax(k) ('size_max') or CountingMax(k) ('counting_max') in one
        contraction (tn_contract_kbest)."""
        import torch
        need = tn_kbest_workspace_bytes(self.handle, kind, k)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_contract_kbest(self.handle, kind, k, workspace.data_ptr(), workspace.numel(), st.cuda_stream)

    def evaluate(self, primes, xs, workspace=None, stream=None) -> list:
        """I(G, xs[q]) mod primes[q] for every slot (tn_contract_modp_x)."""
        import torch
        need = self.workspace_bytes("modp", len(primes))
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_contract_modp_x(self.handle, primes, xs, workspace.data_ptr(), workspace.numel(), st.cuda_stream)

    def independence_polynomial(self, primes=None, degree=None, workspace=None, stream=None) -> list:
        """Exact coefficients of I(G, x) (tn_independence_polynomial).  degree
        defaults to the MIS size from a tropical contraction; primes default
        to the fewest 31-bit primes whose product exceeds 2^n."""
        import torch
        if degree is None:
            degree = self.contract("tropical_i32", workspace=workspace, stream=stream)["max"] or 0
        if primes is None:
            k, prod = 0, 1
            while prod <= (1 << self.n):
                k += 1
                prod *= primes31(k)[-1]
            primes = primes31(k)
        slots = min(TN_MAX_PRIMES, len(primes) * (int(degree) + 1))
        need = self.workspace_bytes("modp", slots)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        coeffs, _ = tn_independence_polynomial(self.handle, primes, degree, workspace.data_ptr(), workspace.numel(),
                                               st.cuda_stream)
        return coeffs

    def contract_weighted(self, semiring, problem, edge_w=None, vertex_w=None, primes=None, xs=None,
                          workspace=None, stream=None) -> dict:
        """Weighted IS ("is") or spin-glass ("spin") contraction (tn_contract_weighted)."""
        import torch
        k = len(primes) if primes is not None else 1
        need = tn_weighted_workspace_bytes(self.handle, semiring, k)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_contract_weighted(self.handle, semiring, problem, edge_w, vertex_w, primes, xs,
                                    workspace.data_ptr(), workspace.numel(), st.cuda_stream)

    def weighted_polynomial(self, problem, edge_w=None, vertex_w=None, primes=None, degree=None,
                            workspace=None, stream=None) -> list:
        """Exact generating polynomial of a weighted network
        (tn_weighted_polynomial).  degree defaults to its largest possible
        value (sum of the weights; 2 (sum|J| + sum|h|) for the spin glass);
        primes to the fewest 31-bit primes whose product exceeds 2^n."""
        import torch
        m = len(self.edges)
        if degree is None:
            if _problem(problem) == TN_PROBLEM_SPIN_GLASS:
                sj = m if edge_w is None else int(np.abs(np.asarray(edge_w, dtype=np.int64)).sum())
                sh = 0 if vertex_w is None else int(np.abs(np.asarray(vertex_w, dtype=np.int64)).sum())
                degree = 2 * (sj + sh)
            else:
                degree = self.n if vertex_w is None else int(np.asarray(vertex_w, dtype=np.int64).sum())
        if primes is None:
            k, prod = 0, 1
            while prod <= (1 << self.n):
                k += 1
                prod *= primes31(k)[-1]
            primes = primes31(k)
        slots = min(TN_MAX_PRIMES, len(primes) * (int(degree) + 1))
        need = tn_weighted_workspace_bytes(self.handle, "modp", slots)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        coeffs, _ = tn_weighted_polynomial(self.handle, problem, edge_w, vertex_w, primes, degree,
                                           workspace.data_ptr(), workspace.numel(), st.cuda_stream)
        return coeffs

    def contract_sliced(self, semiring, problem="is", edge_w=None, vertex_w=None, primes=None, xs=None,
                        slices=None, batch: int = 1, workspace=None, stream=None) -> dict:
        """Sum of the slices in range `slices` (default: all) in the element
        type (tn_contract_sliced), with a workspace for `batch` slices per
        launch."""
        import torch
        nsl = 1 << (0 if self.sliced is None else len(self.sliced))
        b, e = (0, nsl) if slices is None else (int(slices[0]), int(slices[1]))
        k = len(primes) if primes is not None else 1
        need = tn_sliced_workspace_bytes(self.handle, semiring, k, batch)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_contract_sliced(self.handle, semiring, problem, edge_w, vertex_w, primes, xs, b, e,
                                  workspace.data_ptr(), workspace.numel(), st.cuda_stream)

    def single_config_max(self, problem="is", edge_w=None, vertex_w=None, workspace=None, stream=None):
        """(maximum, one configuration reaching it) (tn_single_config_max)."""
        import torch
        need = tn_single_config_workspace_bytes(self.handle)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        return tn_single_config_max(self.handle, problem, edge_w, vertex_w, self.n, workspace.data_ptr(),
                                    workspace.numel(), st.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            tn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many plans contracted in one persistent launch (tn_batch_*)."""

    def __init__(self, plans, semiring, primes=None):
        self.plans = list(plans)
        self.semiring = semiring
        self.primes = primes
        self.handle = tn_batch_create(self.plans, semiring, primes)
        self.info = tn_batch_info(self.handle)
        self.ws = None
        self.raw = None

    def buffers(self):
        import torch
        if self.ws is None:
            self.ws = torch.empty(max(self.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
            self.raw = torch.zeros(len(self.plans) * TN_RAW_BYTES, dtype=torch.uint8, device="cuda")
        return self.ws, self.raw

    def launch(self, graph: bool = False, stream=None):
        """Enqueue the batch (no wait)."""
        import torch
        ws, raw = self.buffers()
        st = (stream or torch.cuda.current_stream()).cuda_stream
        f = tn_batch_contract_graph if graph else tn_batch_contract
        f(self.handle, ws.data_ptr(), ws.numel(), st, raw.data_ptr())

    def results(self):
        import torch
        torch.cuda.current_stream().synchronize()
        host = self.raw.cpu().numpy().tobytes()
        return [tn_result_decode(self.semiring, self.primes, host[i * TN_RAW_BYTES:(i + 1) * TN_RAW_BYTES])
                for i in range(len(self.plans))]

    def run(self, graph: bool = False):
        self.launch(graph)
        return self.results()

    def close(self):
        if getattr(self, "handle", None):
            tn_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

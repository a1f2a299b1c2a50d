"""ctypes binding of the CCM C ABI (include/ccm.h), same names, marshalling only.

Every step of the computation runs in ``libccm_gb300.so``; this module only
converts arguments.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA; a CUDA tensor passes its device pointer, which requires the
plan's ``CCM_INPUT_ON_DEVICE`` / ``CCM_OUTPUT_ON_DEVICE`` flags).  Streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or None.

Importing this module loads the shared library and raises if it has not been
built (``python -c "import __graft_entry__ as g; g.build()"``); there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccm_gb300.so")

CCM_OK = 0
CCM_PENDING = 1
CCM_EINVAL = -1
CCM_ENOMEM = -2
CCM_ETOOLARGE = -3
CCM_ECUDA = -4
CCM_ETIMEOUT = -5
CCM_ECANCELLED = -6
CCM_ENOTFOUND = -7
CCM_INPUT_ON_DEVICE = 0x1
CCM_OUTPUT_ON_DEVICE = 0x2
CCM_NO_AUTOTUNE = 0x4
CCM_NO_TABLE = 0x10
CCM_SEARCH_STATS = 0x20

STATUS_NAMES = {0: "CCM_OK", 1: "CCM_PENDING", -1: "CCM_EINVAL", -2: "CCM_ENOMEM",
                -3: "CCM_ETOOLARGE", -4: "CCM_ECUDA", -5: "CCM_ETIMEOUT",
                -6: "CCM_ECANCELLED", -7: "CCM_ENOTFOUND"}

# Every function the header declares, for the export check.
EXPORTED = ["ccm_context_create", "ccm_context_destroy", "ccm_plan", "ccm_plan_destroy",
            "ccm_plan_get_info", "ccm_run", "ccm_run_ex", "ccm_run_plain", "ccm_submit",
            "ccm_poll", "ccm_cancel", "ccm_job_times", "ccm_last_error", "ccm_version",
            "ccm_plan_kernel_times", "ccm_run_noalloc", "ccm_plan_stage_times",
            "ccm_convergence", "ccm_plan_search_stats"]


class ccm_problem(ctypes.Structure):
    _fields_ = [("n_series", ctypes.c_int32), ("n", ctypes.c_int64),
                ("n_pairs", ctypes.c_int32), ("pairs", ctypes.POINTER(ctypes.c_int32)),
                ("n_E", ctypes.c_int32), ("E", ctypes.POINTER(ctypes.c_int32)),
                ("n_tau", ctypes.c_int32), ("tau", ctypes.POINTER(ctypes.c_int32)),
                ("n_L", ctypes.c_int32), ("L", ctypes.POINTER(ctypes.c_int64)),
                ("r", ctypes.c_int32), ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("theiler", ctypes.c_int32), ("weight_floor", ctypes.c_float)]


class ccm_debug_out(ctypes.Structure):
    _fields_ = [("libraries", ctypes.c_void_p), ("neighbours", ctypes.c_void_p),
                ("predictions", ctypes.c_void_p)]


class ccm_plan_info(ctypes.Structure):
    _fields_ = [("n_units", ctypes.c_int64), ("n_queries", ctypes.c_int64),
                ("library_entries", ctypes.c_int64), ("neighbour_entries", ctypes.c_int64),
                ("n_work_items", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("pair_count", ctypes.c_double), ("flop_count", ctypes.c_double),
                ("brute_flop_count", ctypes.c_double), ("table_bytes", ctypes.c_size_t),
                ("launches_per_run", ctypes.c_int64), ("brute_pair_count", ctypes.c_double),
                ("search_query_count", ctypes.c_int64), ("table_query_count", ctypes.c_int64)]


class ccm_search_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in
                ("brute_tiles", "brute_queries", "pairs_begun", "pairs_full", "pairs_pruned",
                 "candidates", "merge_slots", "table_queries", "table_entries",
                 "table_fallbacks")]


class CCMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library has not been built "
                           "(run `python -c \"import __graft_entry__ as g; g.build()\"`)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    st = ctypes.c_int
    sig = {
        "ccm_context_create": ([ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(vp)], st),
        "ccm_context_destroy": ([vp], st),
        "ccm_plan": ([vp, ctypes.POINTER(ccm_problem), ctypes.POINTER(vp)], st),
        "ccm_plan_destroy": ([vp], st),
        "ccm_plan_get_info": ([vp, ctypes.POINTER(ccm_plan_info)], st),
        "ccm_run": ([vp, vp, vp, vp], st),
        "ccm_run_ex": ([vp, vp, vp, ctypes.POINTER(ccm_debug_out), vp], st),
        "ccm_run_plain": ([vp, vp, vp, vp], st),
        "ccm_plan_kernel_times": ([vp, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)], st),
        "ccm_plan_stage_times": ([vp, ctypes.POINTER(ctypes.c_double)], st),
        "ccm_submit": ([vp, ctypes.POINTER(ccm_problem), vp, ctypes.POINTER(u64)], st),
        "ccm_poll": ([vp, u64, vp, i32], st),
        "ccm_cancel": ([vp, u64], st),
        "ccm_job_times": ([vp, u64, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], st),
        "ccm_run_noalloc": ([vp, i32, i64, i32, i32, i32, i32, i64, i32, u64, vp, vp], st),
        "ccm_convergence": ([vp, vp, i64, i32, vp, i32, ctypes.c_double, vp, ctypes.c_uint32,
                             vp], st),
        "ccm_plan_search_stats": ([vp, ctypes.POINTER(ccm_search_stats)], st),
        "ccm_last_error": ([], ctypes.c_char_p),
        "ccm_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    del i64
    return lib


_lib = _load()


def ccm_last_error() -> str:
    return (_lib.ccm_last_error() or b"").decode()


def ccm_version() -> str:
    return _lib.ccm_version().decode()


def _check(status: int) -> int:
    if status < 0:
        raise CCMError(status, ccm_last_error())
    return status


def _ptr(a, dtype=None) -> int:
    """Address of a C-contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(a.data_ptr())
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot pass {type(a)}")


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


def _problem(series_shape, pairs, E, tau, L, r, seed, flags, keep, theiler=0, weight_floor=0.0):
    pairs = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2))
    E = np.ascontiguousarray(np.asarray(E, np.int32).reshape(-1))
    tau = np.ascontiguousarray(np.asarray(tau, np.int32).reshape(-1))
    L = np.ascontiguousarray(np.asarray(L, np.int64).reshape(-1))
    keep.extend([pairs, E, tau, L])
    V, n = int(series_shape[0]), int(series_shape[1])
    P = ctypes.POINTER
    return ccm_problem(V, n, len(pairs), pairs.ctypes.data_as(P(ctypes.c_int32)),
                       len(E), E.ctypes.data_as(P(ctypes.c_int32)),
                       len(tau), tau.ctypes.data_as(P(ctypes.c_int32)),
                       len(L), L.ctypes.data_as(P(ctypes.c_int64)), int(r), int(seed),
                       int(flags), int(theiler), float(weight_floor))


def ccm_context_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.ccm_context_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
    return h.value


def ccm_context_destroy(ctx: int) -> None:
    _check(_lib.ccm_context_destroy(ctx))


def ccm_plan(ctx: int, series_shape, pairs, E, tau, L, r: int, seed: int, flags: int = 0,
             theiler: int = 0, weight_floor: float = 0.0) -> int:
    keep: list = []
    prob = _problem(series_shape, pairs, E, tau, L, r, seed, flags, keep, theiler, weight_floor)
    h = ctypes.c_void_p()
    _check(_lib.ccm_plan(ctx, ctypes.byref(prob), ctypes.byref(h)))
    return h.value


def ccm_plan_destroy(plan: int) -> None:
    _check(_lib.ccm_plan_destroy(plan))


def ccm_plan_get_info(plan: int) -> dict:
    info = ccm_plan_info()
    _check(_lib.ccm_plan_get_info(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in ccm_plan_info._fields_}


def ccm_run(plan: int, series, rho, stream=None) -> None:
    _check(_lib.ccm_run(plan, _ptr(series), _ptr(rho), _stream(stream)))


def ccm_run_ex(plan: int, series, rho, libraries=None, neighbours=None, predictions=None,
               stream=None) -> None:
    dbg = ccm_debug_out(_ptr(libraries) or None, _ptr(neighbours) or None,
                        _ptr(predictions) or None)
    _check(_lib.ccm_run_ex(plan, _ptr(series), _ptr(rho), ctypes.byref(dbg), _stream(stream)))


def ccm_plan_kernel_times(plan: int):
    """(sampler_ms, knn_ms) device times of the plan's last completed run."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ccm_plan_kernel_times(plan, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ccm_plan_stage_times(plan: int):
    """[order + tables, sampler, brute-force kNN, table-scan kNN] device ms of the last run."""
    out = (ctypes.c_double * 4)()
    _check(_lib.ccm_plan_stage_times(plan, out))
    return list(out)


def ccm_plan_search_stats(plan: int) -> dict:
    """Work counts of the last run of a plan made with CCM_SEARCH_STATS."""
    out = ccm_search_stats()
    _check(_lib.ccm_plan_search_stats(plan, ctypes.byref(out)))
    return {name: int(getattr(out, name)) for name, _ in ccm_search_stats._fields_}


def ccm_run_plain(plan: int, series, rho, stream=None) -> None:
    _check(_lib.ccm_run_plain(plan, _ptr(series), _ptr(rho), _stream(stream)))


def ccm_submit(ctx: int, series, pairs, E, tau, L, r: int, seed: int, theiler: int = 0,
               weight_floor: float = 0.0) -> int:
    keep: list = []
    series = np.ascontiguousarray(series, dtype=np.float32)
    prob = _problem(series.shape, pairs, E, tau, L, r, seed, 0, keep, theiler, weight_floor)
    t = ctypes.c_uint64()
    _check(_lib.ccm_submit(ctx, ctypes.byref(prob), _ptr(series), ctypes.byref(t)))
    return t.value


def ccm_poll(ctx: int, ticket: int, rho, timeout_ms: int = 0) -> int:
    """CCM_OK (rho written) or CCM_PENDING; raises CCMError on a failed job."""
    return _check(_lib.ccm_poll(ctx, int(ticket), _ptr(rho, np.float64), int(timeout_ms)))


def ccm_cancel(ctx: int, ticket: int) -> int:
    return _check(_lib.ccm_cancel(ctx, int(ticket)))


def ccm_job_times(ctx: int, ticket: int):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = _check(_lib.ccm_job_times(ctx, int(ticket), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(c)))
    return st, a.value, b.value, c.value


def ccm_run_noalloc(d_series, j: int, i: int, E: int, tau: int, L: int, r: int, seed: int,
                    d_rho, stream=None) -> None:
    """One cell into device ``d_rho`` [r] from device ``d_series`` [V][n], with no
    device allocation (all scratch in the library's fixed device array)."""
    V, n = int(d_series.shape[0]), int(d_series.shape[1])
    _check(_lib.ccm_run_noalloc(_ptr(d_series), V, n, int(j), int(i), int(E), int(tau), int(L),
                                int(r), int(seed), _ptr(d_rho), _stream(stream)))


def plan_problem(ctx: int, problem, flags: int = 0) -> int:
    """ccm_plan for an object with series, pairs, E, tau, L, r and seed attributes
    (and optionally theiler and weight_floor)."""
    return ccm_plan(ctx, problem.series.shape, problem.pairs, problem.E, problem.tau, problem.L,
                    problem.r, problem.seed, flags, getattr(problem, "theiler", 0),
                    getattr(problem, "weight_floor", 0.0))


def rho_shape(problem) -> tuple:
    return (len(problem.pairs), len(problem.E), len(problem.tau), len(problem.L), int(problem.r))


CONVERGENCE_FIELDS = ("rho_first", "rho_last", "jt", "z", "n_valid", "converged")


class ccm_convergence_t(ctypes.Structure):
    _fields_ = [("rho_first", ctypes.c_double), ("rho_last", ctypes.c_double),
                ("jt", ctypes.c_double), ("z", ctypes.c_double),
                ("n_valid", ctypes.c_int32), ("converged", ctypes.c_int32)]


_CONV_DTYPE = np.dtype([("rho_first", "<f8"), ("rho_last", "<f8"), ("jt", "<f8"), ("z", "<f8"),
                        ("n_valid", "<i4"), ("converged", "<i4")])


def ccm_convergence(ctx: int, rho, L, z_crit: float = 1.6448536269514722, out=None,
                    stream=None):
    """Convergence decision per (pair, E, tau) row of ``rho`` [..., n_L, r] (host
    numpy or device tensor).  Returns a structured numpy array [...] with the
    fields of ccm_convergence_t, or fills ``out`` (device memory of 40 bytes
    per row, e.g. a uint8 tensor) and returns it."""
    L = np.ascontiguousarray(np.asarray(L, np.int64).reshape(-1))
    shape = tuple(rho.shape)
    n_L, r = int(shape[-2]), int(shape[-1])
    if len(L) != n_L:
        raise ValueError("L must match rho's L axis")
    n_rows = int(np.prod(shape[:-2])) if len(shape) > 2 else 1
    on_dev = not isinstance(rho, np.ndarray)
    flags = CCM_INPUT_ON_DEVICE if on_dev else 0
    if out is None:
        host = np.zeros(n_rows, _CONV_DTYPE)
        _check(_lib.ccm_convergence(ctx, _ptr(rho), n_rows, n_L, L.ctypes.data, r,
                                    float(z_crit), host.ctypes.data, flags, _stream(stream)))
        return host.reshape(shape[:-2])
    _check(_lib.ccm_convergence(ctx, _ptr(rho), n_rows, n_L, L.ctypes.data, r, float(z_crit),
                                _ptr(out), flags | CCM_OUTPUT_ON_DEVICE, _stream(stream)))
    return out

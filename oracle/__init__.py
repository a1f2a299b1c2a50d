"""CPU oracle for convergent cross mapping -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded FP64 CCM (``ccm_oracle.cpp``) behind ctypes.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg use it; the CUDA
library never calls, links or imports anything here, and this package imports
nothing from the CUDA side.

Each wrapper names the step of the method it follows; the C++ file cites the
paper's sections.  Neighbour selection is taken on FP32 squared distances by
default (``select_fp64=False``), the precision the GPU kernel decides in, or on
FP64 squared distances (``select_fp64=True``) to measure how often the FP32
decision differs from the FP64 one.  Two options the paper does not discuss,
off by default: an exclusion (Theiler) window ``theiler`` and a weight floor
``weight_floor`` (see ``ccm_oracle.cpp``).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccm_oracle.cpp")
_SO = os.path.join(_HERE, "libccm_oracle.so")
_lock = threading.Lock()
_lib = None

_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_F32P = ctypes.POINTER(ctypes.c_float)
_F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``libccm_oracle.so`` with g++ (no -ffast-math, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_philox4x64_10.argtypes = [_U64P, _U64P, _U64P]
            lib.oracle_philox4x64_10.restype = None
            lib.oracle_library.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_uint64, _I32P]
            lib.oracle_library.restype = ctypes.c_int
            lib.oracle_neighbours.argtypes = [_F32P, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, _I32P, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int32, _I32P]
            lib.oracle_neighbours.restype = ctypes.c_int
            lib.oracle_predict.argtypes = [_F32P, _F32P, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, _I32P, _F64P]
            lib.oracle_predict.restype = ctypes.c_int
            lib.oracle_query_subset.argtypes = [_F32P, _F32P, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_int32, _I32P, ctypes.c_int64, _I64P,
                                                ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_double, _I32P, _F64P]
            lib.oracle_query_subset.restype = ctypes.c_int
            lib.oracle_query_margin.argtypes = [_F32P, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_int32, _I32P, ctypes.c_int64, _I64P,
                                                ctypes.c_int64, ctypes.c_int32, _F64P]
            lib.oracle_query_margin.restype = ctypes.c_int
            lib.oracle_pearson.argtypes = [_F64P, _F64P, ctypes.c_int64]
            lib.oracle_pearson.restype = ctypes.c_double
            lib.oracle_skill.argtypes = [_F32P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         _F64P]
            lib.oracle_skill.restype = ctypes.c_double
            lib.oracle_ccm_unit.argtypes = [_F32P, ctypes.c_int32, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_double, _F64P, _I32P, _I32P, _F64P]
            lib.oracle_ccm_unit.restype = ctypes.c_int
            lib.oracle_ccm.argtypes = [_F32P, ctypes.c_int32, ctypes.c_int64, _I32P,
                                       ctypes.c_int32, _I32P, ctypes.c_int32, _I32P,
                                       ctypes.c_int32, _I64P, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, _F64P]
            lib.oracle_ccm.restype = ctypes.c_int
            lib.oracle_convergence.argtypes = [_F64P, ctypes.c_int64, ctypes.c_int32, _I64P,
                                               ctypes.c_int32, ctypes.c_double, _F64P]
            lib.oracle_convergence.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def philox4x64_10(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for a 4-word counter and 2-word key (uint64[4])."""
    c = _c(ctr, np.uint64)
    k = _c(key, np.uint64)
    out = np.zeros(4, np.uint64)
    _load().oracle_philox4x64_10(_ptr(c, _U64P), _ptr(k, _U64P), _ptr(out, _U64P))
    return out


def library(n_m: int, L: int, j: int, E: int, tau: int, k: int, seed: int) -> np.ndarray:
    """Library of one realization: L ascending manifold indices (int32)."""
    out = np.zeros(int(L), np.int32)
    rc = _load().oracle_library(int(n_m), int(L), int(j), int(E), int(tau), int(k),
                                int(seed), _ptr(out, _I32P))
    if rc != 0:
        raise ValueError("invalid library size")
    return out


def neighbours(s: np.ndarray, E: int, tau: int, lib: np.ndarray,
               select_fp64: bool = False, theiler: int = 0) -> np.ndarray:
    """E+1 nearest library neighbours [N_m][E+1] of every manifold point of ``s``;
    candidates of query m are the library points l with |l - m| > theiler."""
    s = _c(s, np.float32)
    lib = _c(lib, np.int32)
    n_m = len(s) - (E - 1) * tau
    out = np.zeros((n_m, E + 1), np.int32)
    rc = _load().oracle_neighbours(_ptr(s, _F32P), len(s), int(E), int(tau), _ptr(lib, _I32P),
                                   len(lib), int(bool(select_fp64)), int(theiler),
                                   _ptr(out, _I32P))
    if rc != 0:
        raise ValueError("invalid neighbour search arguments")
    return out


def predict(lib_s: np.ndarray, tgt_s: np.ndarray, E: int, tau: int,
            nbr: np.ndarray, weight_floor: float = 0.0) -> np.ndarray:
    """Simplex predictions Xhat [N_m] (FP64) from neighbour lists [N_m][E+1];
    u_i = max(exp(-d_i/d_1), weight_floor)."""
    lib_s = _c(lib_s, np.float32)
    tgt_s = _c(tgt_s, np.float32)
    nbr = _c(nbr, np.int32)
    n_m = len(lib_s) - (E - 1) * tau
    assert nbr.shape == (n_m, E + 1)
    out = np.zeros(n_m, np.float64)
    rc = _load().oracle_predict(_ptr(lib_s, _F32P), _ptr(tgt_s, _F32P), len(lib_s), int(E),
                                int(tau), float(weight_floor), _ptr(nbr, _I32P),
                                _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("invalid prediction arguments")
    return out


def query_subset(lib_s: np.ndarray, tgt_s: np.ndarray, E: int, tau: int, lib: np.ndarray,
                 queries, select_fp64: bool = False, theiler: int = 0,
                 weight_floor: float = 0.0):
    """Neighbours [nq][E+1] and predictions [nq] of the listed query points only."""
    lib_s = _c(lib_s, np.float32)
    tgt_s = _c(tgt_s, np.float32)
    lib = _c(lib, np.int32)
    q = _c(queries, np.int64)
    nbr = np.zeros((len(q), E + 1), np.int32)
    xh = np.zeros(len(q), np.float64)
    rc = _load().oracle_query_subset(_ptr(lib_s, _F32P), _ptr(tgt_s, _F32P), len(lib_s), int(E),
                                     int(tau), _ptr(lib, _I32P), len(lib), _ptr(q, _I64P), len(q),
                                     int(bool(select_fp64)), int(theiler), float(weight_floor),
                                     _ptr(nbr, _I32P), _ptr(xh, _F64P))
    if rc != 0:
        raise ValueError("invalid query subset arguments")
    return nbr, xh


def query_margin(s: np.ndarray, E: int, tau: int, lib: np.ndarray, queries,
                 theiler: int = 0) -> np.ndarray:
    """Per listed query, the relative FP64 gap (d_b - d_a) / d_b between its
    (E+1)-th and (E+2)-th nearest candidate distances (inf with only E+1
    candidates, 0 when d_b = 0): a neighbour set chosen in FP32 may differ
    from the FP64 one only where this gap is small."""
    s = _c(s, np.float32)
    lib = _c(lib, np.int32)
    q = _c(queries, np.int64)
    out = np.zeros(len(q), np.float64)
    rc = _load().oracle_query_margin(_ptr(s, _F32P), len(s), int(E), int(tau), _ptr(lib, _I32P),
                                     len(lib), _ptr(q, _I64P), len(q), int(theiler),
                                     _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("invalid margin arguments")
    return out


def pearson(x: np.ndarray, y: np.ndarray) -> float:
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    return float(_load().oracle_pearson(_ptr(x, _F64P), _ptr(y, _F64P), len(x)))


def skill(tgt_s: np.ndarray, E: int, tau: int, xhat: np.ndarray) -> float:
    """Pearson rho between the observed target at t_m and the predictions."""
    tgt_s = _c(tgt_s, np.float32)
    xhat = _c(xhat, np.float64)
    return float(_load().oracle_skill(_ptr(tgt_s, _F32P), len(tgt_s), int(E), int(tau),
                                      _ptr(xhat, _F64P)))


def ccm_unit(series: np.ndarray, j: int, i: int, E: int, tau: int, L: int, k: int, seed: int,
             select_fp64: bool = False, keep: bool = False, theiler: int = 0,
             weight_floor: float = 0.0):
    """rho of one unit; with ``keep`` also (library, neighbours, Xhat)."""
    series = _c(series, np.float32)
    V, n = series.shape
    n_m = n - (E - 1) * tau
    rho = np.zeros(1, np.float64)
    lib = np.zeros(int(L), np.int32) if keep else None
    nbr = np.zeros((max(n_m, 0), E + 1), np.int32) if keep else None
    xh = np.zeros(max(n_m, 0), np.float64) if keep else None
    rc = _load().oracle_ccm_unit(
        _ptr(series, _F32P), V, n, int(j), int(i), int(E), int(tau), int(L), int(k), int(seed),
        int(bool(select_fp64)), int(theiler), float(weight_floor), _ptr(rho, _F64P),
        _ptr(lib, _I32P) if keep else None, _ptr(nbr, _I32P) if keep else None,
        _ptr(xh, _F64P) if keep else None)
    if rc != 0:
        raise ValueError("invalid CCM unit")
    if keep:
        return float(rho[0]), lib, nbr, xh
    return float(rho[0])


def ccm(series, pairs, E, tau, L, r: int, seed: int, select_fp64: bool = False,
        theiler: int = 0, weight_floor: float = 0.0) -> np.ndarray:
    """Whole sweep: rho [n_pairs][n_E][n_tau][n_L][r] (FP64)."""
    series = _c(series, np.float32)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    E = _c(E, np.int32)
    tau = _c(tau, np.int32)
    L = _c(L, np.int64)
    V, n = series.shape
    out = np.zeros((len(pairs), len(E), len(tau), len(L), int(r)), np.float64)
    rc = _load().oracle_ccm(_ptr(series, _F32P), V, n, _ptr(pairs, _I32P), len(pairs),
                            _ptr(E, _I32P), len(E), _ptr(tau, _I32P), len(tau), _ptr(L, _I64P),
                            len(L), int(r), int(seed), int(bool(select_fp64)), int(theiler),
                            float(weight_floor), _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("invalid CCM problem")
    return out


def convergence(rho, L, z_crit: float = 1.6448536269514722) -> np.ndarray:
    """Convergence decision per (pair, E, tau) row of rho [..., n_L, r]: an array
    [..., 6] of (mean rho at the smallest L, at the largest L, Jonckheere-Terpstra
    J, its z score, finite realizations, converged 0/1).  Default z_crit: the
    one-sided 5% point of the standard normal."""
    rho = _c(rho, np.float64)
    L = _c(L, np.int64)
    n_L, r = rho.shape[-2], rho.shape[-1]
    assert len(L) == n_L
    rows = rho.reshape(-1, n_L, r)
    out = np.zeros((rows.shape[0], 6), np.float64)
    rc = _load().oracle_convergence(_ptr(rows, _F64P), rows.shape[0], n_L, _ptr(L, _I64P), r,
                                    float(z_crit), _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("invalid convergence arguments")
    return out.reshape(rho.shape[:-2] + (6,))

"""FP64 CPU oracle for PALMAD discord discovery -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, optional OpenMP); this
module compiles it on first use and exposes numpy-friendly wrappers.  See the
header of ``oracle.c`` for the paper passages each function follows and the
readings taken where the paper is ambiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_stats.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _f64p, _f64p]
            lib.oracle_dist.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_dist.restype = ctypes.c_double
            lib.oracle_mp.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _f64p, _i64p]
            lib.oracle_nn_one.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _f64p, _i64p]
            lib.oracle_range_discords.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _i64p,
                                                  _f64p, ctypes.c_int64, _i64p]
            lib.oracle_range_discord_windows.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                                         _i64p, ctypes.c_int64, _f64p]
            lib.oracle_topk.argtypes = [_i64p, _f64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                        _i64p, _f64p]
            lib.oracle_merlin.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int, _i64p, _f64p, _i64p, _f64p, _i32p, _f32p]
            lib.oracle_knn.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _f64p]
            lib.oracle_drag_knn.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                            _f64p, _i64p, _f64p, ctypes.c_int64, _i64p]
            lib.oracle_merlin_knn.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int, ctypes.c_int32, _i64p, _f64p, _i64p, _f64p, _i32p, _f32p]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f32(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, dtype=np.float32))


def _p(a, t):
    return a.ctypes.data_as(t)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def stats(T, m: int):
    """Per-window mean and population standard deviation (Eq. 4), FP64."""
    T = _f32(T)
    N = len(T) - m + 1
    mu, sd = np.empty(N), np.empty(N)
    rc = _load().oracle_stats(_p(T, _f32p), len(T), m, _p(mu, _f64p), _p(sd, _f64p))
    if rc:
        raise ValueError(f"oracle_stats rc={rc}")
    return mu, sd


def dist(T, m: int, i: int, j: int) -> float:
    """z-normalised Euclidean distance between windows i and j (Eq. 4-5)."""
    T = _f32(T)
    return float(_load().oracle_dist(_p(T, _f32p), len(T), m, i, j))


def matrix_profile(T, m: int):
    """Brute-force nearest non-self-match distance and index of every window."""
    T = _f32(T)
    N = len(T) - m + 1
    mp, idx = np.empty(N), np.empty(N, dtype=np.int64)
    rc = _load().oracle_mp(_p(T, _f32p), len(T), m, _p(mp, _f64p), _p(idx, _i64p))
    if rc:
        raise ValueError(f"oracle_mp rc={rc}")
    return mp, idx


def nn_one(T, m: int, i: int):
    """Brute-force nearest non-self match of window i: (distance, index)."""
    T = _f32(T)
    nn, idx = ctypes.c_double(0.0), ctypes.c_int64(0)
    rc = _load().oracle_nn_one(_p(T, _f32p), len(T), m, i, ctypes.byref(nn), ctypes.byref(idx))
    if rc:
        raise ValueError(f"oracle_nn_one rc={rc}")
    return nn.value, idx.value


def knn_profile(T, m: int, k: int):
    """k-distance of every window (reading R14): the k-th smallest distance
    to its non-self matches, by brute force; inf where a window has fewer
    than k non-self matches."""
    T = _f32(T)
    out = np.empty(len(T) - m + 1)
    rc = _load().oracle_knn(_p(T, _f32p), len(T), m, k, _p(out, _f64p))
    if rc:
        raise ValueError(f"oracle_knn rc={rc}")
    return out


def drag_knn(T, m: int, k: int, r: float, profile=None):
    """Range k-discords of length m at threshold r (reading R14): ascending
    indices and their k-distances.  `profile` may pass the k-distances from
    knn_profile(T, m, k) so that they are not recomputed."""
    T = _f32(T)
    prof = None
    if profile is not None:
        prof = np.ascontiguousarray(profile, dtype=np.float64)
        if len(prof) != len(T) - m + 1:
            raise ValueError("profile length must be n - m + 1")
    cap = 1024
    while True:
        idx, nn = np.empty(cap, dtype=np.int64), np.empty(cap)
        cnt = ctypes.c_int64(0)
        rc = _load().oracle_drag_knn(_p(T, _f32p), len(T), m, k, float(r), _p(prof, _f64p) if prof is not None else None,
                                     _p(idx, _i64p), _p(nn, _f64p), cap, ctypes.byref(cnt))
        if rc:
            raise ValueError(f"oracle_drag_knn rc={rc}")
        if cnt.value <= cap:
            return idx[:cnt.value].copy(), nn[:cnt.value].copy()
        cap = cnt.value


def range_discords(T, m: int, r: float):
    """All range discords of length m at threshold r (Sec. 2.1), the set one
    DRAG call (Algorithm 2) returns: ascending indices and their
    nearest-neighbour distances."""
    T = _f32(T)
    cap = 1024
    while True:
        idx, nn = np.empty(cap, dtype=np.int64), np.empty(cap)
        cnt = ctypes.c_int64(0)
        rc = _load().oracle_range_discords(_p(T, _f32p), len(T), m, float(r), _p(idx, _i64p), _p(nn, _f64p), cap,
                                           ctypes.byref(cnt))
        if rc:
            raise ValueError(f"oracle_range_discords rc={rc}")
        if cnt.value <= cap:
            return idx[:cnt.value].copy(), nn[:cnt.value].copy()
        cap = cnt.value


def range_discord_windows(T, m: int, r: float, windows):
    """The range-discord test of Sec. 2.1 for the listed windows only: per
    window its nnDist when it is a range discord at r, NaN otherwise."""
    T = _f32(T)
    w = np.ascontiguousarray(windows, dtype=np.int64)
    out = np.empty(len(w))
    rc = _load().oracle_range_discord_windows(_p(T, _f32p), len(T), m, float(r), _p(w, _i64p), len(w),
                                              _p(out, _f64p))
    if rc:
        raise ValueError(f"oracle_range_discord_windows rc={rc}")
    return out


# The output of one DRAG call at (m, r): the name the parity tests use.
drag = range_discords


def topk(idx, nn, m: int, K: int, exclusive: bool = True):
    """Greedy top-K of (index, nnDist) pairs; -1 / 0.0 pad when fewer."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    nn = np.ascontiguousarray(nn, dtype=np.float64)
    oi, on = np.empty(K, dtype=np.int64), np.empty(K)
    got = _load().oracle_topk(_p(idx, _i64p), _p(nn, _f64p), len(idx), m, K, int(exclusive),
                              _p(oi, _i64p), _p(on, _f64p))
    if got < 0:
        raise ValueError(f"oracle_topk rc={got}")
    return oi, on


def interest(heat, minL: int, K: int, exclusive: bool = True):
    """Eq. 11: per-index interest (largest heatmap value over the lengths)
    and its length, and the greedy top-K interesting discords.  Returns a
    dict with ``score`` [W], ``best_m`` [W], ``idx`` [K], ``m`` [K],
    ``value`` [K] (-1 / 0 / 0 past the last pick)."""
    heat = np.ascontiguousarray(heat, dtype=np.float32)
    L, W = heat.shape
    out = {"score": np.empty(W, dtype=np.float32), "best_m": np.empty(W, dtype=np.int32),
           "idx": np.empty(K, dtype=np.int64), "m": np.empty(K, dtype=np.int32), "value": np.empty(K, dtype=np.float32)}
    got = _load().oracle_interest(_p(heat, _f32p), L, W, minL, K, int(exclusive), _p(out["score"], _f32p),
                                  _p(out["best_m"], _i32p), _p(out["idx"], _i64p), _p(out["m"], _i32p),
                                  _p(out["value"], _f32p))
    if got < 0:
        raise ValueError(f"oracle_interest rc={got}")
    return out


def merlin(T, minL: int, maxL: int, K: int, exclusive: bool = True, heatmap: bool = False, knn: int = 1):
    """MERLIN over lengths minL..maxL (Sec. 2.2; Algorithm 1).  Returns a dict with
    ``idx`` [L,K], ``nn`` [L,K], ``count`` [L], ``r`` [L], ``calls`` [L] and,
    when asked, ``heatmap`` [L, n-minL+1].  knn > 1 runs it on the k-th
    neighbour distance (reading R14) instead of the nearest one."""
    T = _f32(T)
    L = maxL - minL + 1
    out = {
        "idx": np.empty((L, K), dtype=np.int64), "nn": np.empty((L, K)),
        "count": np.empty(L, dtype=np.int64), "r": np.empty(L), "calls": np.empty(L, dtype=np.int32),
    }
    heat = np.empty((L, len(T) - minL + 1), dtype=np.float32) if heatmap else None
    rc = _load().oracle_merlin_knn(_p(T, _f32p), len(T), minL, maxL, K, int(exclusive), int(knn),
                                   _p(out["idx"], _i64p), _p(out["nn"], _f64p), _p(out["count"], _i64p),
                                   _p(out["r"], _f64p), _p(out["calls"], _i32p),
                                   _p(heat, _f32p) if heat is not None else None)
    if rc:
        raise ValueError(f"oracle_merlin rc={rc}")
    if heat is not None:
        out["heatmap"] = heat
    return out

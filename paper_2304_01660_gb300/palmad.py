"""Thin ctypes binding of libpalmad.so (include/palmad.h).

Argument marshalling only: every step of discord discovery runs in the CUDA
library.  Loading fails loudly when the library is missing -- there is no CPU
fallback.  Host arrays are numpy; the ``*_device`` entry takes torch CUDA
tensors (torch serves as the device-memory allocator only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpalmad.so")

PALMAD_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_NONFINITE", -3: "ERR_OOM", -4: "ERR_CUDA", -5: "ERR_TIMEOUT",
          -6: "ERR_UNSUPPORTED", -7: "ERR_INTERNAL", -8: "ERR_TOO_LARGE"}
NOALLOC_MAX_WINDOWS = 1 << 18
PREC_FP32, PREC_MIXED = 0, 1
KERNELS = ["stats", "select", "compact", "plan", "refine_sweep", "refine_direct", "recheck", "gather", "topk", "heat",
           "hint", "seed_tc"]


class PalmadError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("exclusive_topk", ctypes.c_int32),
        ("batch_lengths", ctypes.c_int32),
        ("band_rel", ctypes.c_double),
        ("select_cap", ctypes.c_int32),
        ("reserved_a", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("pool_slots", ctypes.c_int32),
        ("direct_below", ctypes.c_int32),
        ("tc_seed_min", ctypes.c_int32),
        ("seed_rows_max", ctypes.c_int32),
        ("refine_seg", ctypes.c_int32),
        ("knn_k", ctypes.c_int32),
        ("no_hints", ctypes.c_int32),
        ("spec_scale", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("refine_rows", ctypes.c_int32),
        ("direct_below_long", ctypes.c_int32),
        ("tc_group", ctypes.c_int32),
        ("tc_chunks", ctypes.c_int32),
        ("tc_form", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("lengths", ctypes.c_int32),
        ("drag_calls", ctypes.c_int64),
        ("device_passes", ctypes.c_int64),
        ("reruns", ctypes.c_int64),
        ("select_pairs", ctypes.c_int64),
        ("refine_pairs", ctypes.c_int64),
        ("fp64_pairs", ctypes.c_int64),
        ("survivors", ctypes.c_int64),
        ("discords", ctypes.c_int64),
        ("max_fp32_rho_err", ctypes.c_double),
        ("select_flops", ctypes.c_double),
        ("refine_flops", ctypes.c_double),
        ("sweep_flops", ctypes.c_double),
        ("launches", ctypes.c_int64 * 12),
        ("kernel_ms", ctypes.c_double * 12),
        ("seed_pairs", ctypes.c_int64),
        ("seed_flops", ctypes.c_double),
        ("hint_pairs", ctypes.c_int64),
        ("hint_kills", ctypes.c_int64),
        ("refine_strips", ctypes.c_int64),
        ("sweep_survivors", ctypes.c_int64),
        ("tune_ms", ctypes.c_double),
        ("direct_pairs", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("launches", "kernel_ms", "struct_size")}
        d["launches"] = {KERNELS[i]: int(self.launches[i]) for i in range(12)}
        d["kernel_ms"] = {KERNELS[i]: float(self.kernel_ms[i]) for i in range(12)}
        return d


class TuneReport(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("candidates", ctypes.c_int32),
        ("block_lo", ctypes.c_int32),
        ("block_hi", ctypes.c_int32),
        ("tune_ms", ctypes.c_double),
        ("best_ms", ctypes.c_double),
        ("default_ms", ctypes.c_double),
    ]


TUNED_FIELDS = ("batch_lengths", "spec_scale", "select_cap", "refine_seg", "direct_below", "direct_below_long",
                "refine_rows", "tc_chunks")

_lib = None
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH):
    """Load libpalmad.so (raises if it is missing or does not load)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpalmad.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    lib.palmad_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.palmad_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp]
    lib.palmad_destroy.argtypes = [_vp]
    lib.palmad_destroy.restype = None
    lib.palmad_last_error.argtypes = [_vp]
    lib.palmad_last_error.restype = ctypes.c_char_p
    lib.palmad_version.restype = ctypes.c_char_p
    lib.palmad_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
    lib.palmad_find_discords.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(Options), _vp, _vp, _vp, _vp, _vp]
    lib.palmad_find_discords_device.argtypes = lib.palmad_find_discords.argtypes
    lib.palmad_find_discords_resume.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Options), _vp, _vp,
                                                _vp, _vp, _vp, _vp]
    lib.palmad_find_discords_batch.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_int32,
                                               ctypes.POINTER(Options), _vp, _vp, _vp, _vp]
    lib.palmad_drag.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                ctypes.POINTER(Options), _vp, _vp, ctypes.c_int64, _i64p]
    lib.palmad_topk_profile_noalloc.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                                ctypes.c_int32, _vp, _vp, _vp, _vp]
    lib.palmad_schedule_inputs.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp]
    lib.palmad_drag_select_shard.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(Options), _vp]
    lib.palmad_drag_refine_shard.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _vp,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(Options), _vp]
    lib.palmad_autotune.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(Options), ctypes.POINTER(Options), ctypes.POINTER(TuneReport)]
    lib.palmad_measure_peak.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    lib.palmad_discord_interest.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]
    for name in ("palmad_default_options", "palmad_create", "palmad_get_stats", "palmad_find_discords",
                 "palmad_find_discords_device", "palmad_find_discords_batch", "palmad_drag",
                 "palmad_topk_profile_noalloc", "palmad_measure_peak", "palmad_discord_interest",
                 "palmad_find_discords_resume", "palmad_autotune", "palmad_drag_select_shard",
                 "palmad_drag_refine_shard", "palmad_schedule_inputs"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def palmad_version() -> str:
    return load().palmad_version().decode()


def palmad_default_options(**kw) -> Options:
    o = Options()
    load().palmad_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def palmad_topk_profile_noalloc(nn_dev, m: int, r: float, K: int, exclusive: bool = True, stream=None):
    """Top-K range discords of a device profile (float64 CUDA tensor) with no
    allocation inside the library; the output tensors are allocated here by
    torch, on the caller's side.  Returns (idx, nn, count) CUDA tensors,
    ready once `stream` (default: torch's current stream) reaches them."""
    import torch
    assert nn_dev.is_cuda and nn_dev.dtype == torch.float64 and nn_dev.is_contiguous()
    dev = nn_dev.device
    idx = torch.empty(K, dtype=torch.int64, device=dev)
    nn = torch.empty(K, dtype=torch.float64, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    with torch.cuda.device(dev):  # the entry runs on (and caches its scratch address for) the current device
        st = load().palmad_topk_profile_noalloc(nn_dev.data_ptr(), nn_dev.numel(), m, float(r), K,
                                                int(bool(exclusive)), idx.data_ptr(), nn.data_ptr(),
                                                cnt.data_ptr(), s)
    if st != PALMAD_OK:
        raise PalmadError(st, "palmad_topk_profile_noalloc failed")
    return idx, nn, cnt


def palmad_discord_interest(heat_dev, minL: int, K: int, exclusive: bool = True, stream=None) -> dict:
    """Eq. 11 on a device heatmap (float32 CUDA tensor [L, W]): per-index
    interest and length, and the top-K interesting discords.  Returns CUDA
    tensors ``score`` [W], ``best_m`` [W], ``idx`` [K], ``m`` [K], ``value`` [K]."""
    import torch
    assert heat_dev.is_cuda and heat_dev.dtype == torch.float32 and heat_dev.is_contiguous() and heat_dev.dim() == 2
    L, W = heat_dev.shape
    dev = heat_dev.device
    out = {"score": torch.empty(W, dtype=torch.float32, device=dev), "best_m": torch.empty(W, dtype=torch.int32, device=dev),
           "idx": torch.empty(K, dtype=torch.int64, device=dev), "m": torch.empty(K, dtype=torch.int32, device=dev),
           "value": torch.empty(K, dtype=torch.float32, device=dev)}
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    st = load().palmad_discord_interest(heat_dev.data_ptr(), L, W, minL, K, int(bool(exclusive)),
                                        out["score"].data_ptr(), out["best_m"].data_ptr(), out["idx"].data_ptr(),
                                        out["m"].data_ptr(), out["value"].data_ptr(), s)
    if st != PALMAD_OK:
        raise PalmadError(st, "palmad_discord_interest failed")
    return out


def schedule_inputs(idx, nn) -> np.ndarray:
    """palmad_schedule_inputs: per length, the value the schedule carries to
    the next lengths (idx / nn: [L, K] results).  A checkpoint at length m0
    of a run that started at minL is schedule_inputs(...)[max(0, l0 - 5):l0],
    l0 = m0 - minL."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    nn = np.ascontiguousarray(nn, dtype=np.float64)
    L, K = idx.shape
    out = np.empty(L, dtype=np.float64)
    st = load().palmad_schedule_inputs(_ptr(idx), _ptr(nn), L, K, _ptr(out))
    if st != PALMAD_OK:
        raise PalmadError(st, "palmad_schedule_inputs failed")
    return out


PEAK_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def palmad_measure_peak(device: int = 0, kind: str = "fp32") -> float:
    """Measured FMA throughput of `device` in TFLOP/s (kind: fp32, fp32x2
    or fp64)."""
    v = ctypes.c_double(0.0)
    st = load().palmad_measure_peak(device, PEAK_KINDS[kind], ctypes.byref(v))
    if st != PALMAD_OK:
        raise PalmadError(st, "palmad_measure_peak failed")
    return v.value


def _ptr(a) -> int:
    return a.ctypes.data if a is not None else None


class Context:
    """A palmad_ctx on one CUDA device (palmad_create / palmad_destroy)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._lib = load()
        self._h = _vp()
        st = self._lib.palmad_create(ctypes.byref(self._h), device, stream)
        if st != PALMAD_OK:
            raise PalmadError(st, "palmad_create failed")

    def close(self):
        if self._h:
            self._lib.palmad_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != PALMAD_OK:
            raise PalmadError(st, self._lib.palmad_last_error(self._h).decode())

    def palmad_last_error(self) -> str:
        return self._lib.palmad_last_error(self._h).decode()

    def palmad_get_stats(self) -> dict:
        s = Stats()
        s.struct_size = ctypes.sizeof(Stats)
        self._check(self._lib.palmad_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def palmad_find_discords(self, T, minL: int, maxL: int, topK: int, options: Options | None = None,
                             heatmap: bool = False, heat_out=None) -> dict:
        """Host-memory MERLIN over one series; see palmad_find_discords in palmad.h.
        heat_out: optional float32 [L, n - minL + 1] array (e.g. pinned) the
        heatmap is written into."""
        T = np.ascontiguousarray(T, dtype=np.float32)
        L = maxL - minL + 1
        idx = np.empty((L, topK), dtype=np.int64)
        nn = np.empty((L, topK), dtype=np.float64)
        cnt = np.empty(L, dtype=np.int64)
        rr = np.empty(L, dtype=np.float64)
        heat = None
        if heatmap:
            shape = (L, len(T) - minL + 1)
            if heat_out is not None:
                if heat_out.shape != shape or heat_out.dtype != np.float32 or not heat_out.flags.c_contiguous:
                    raise ValueError(f"heat_out must be a C-contiguous float32 array of shape {shape}")
                heat = heat_out
            else:
                heat = np.empty(shape, dtype=np.float32)
        self._check(self._lib.palmad_find_discords(
            self._h, _ptr(T), len(T), minL, maxL, topK, ctypes.byref(options) if options else None,
            _ptr(idx), _ptr(nn), _ptr(cnt), _ptr(rr), _ptr(heat)))
        out = {"idx": idx, "nn": nn, "count": cnt, "r": rr}
        if heat is not None:
            out["heatmap"] = heat
        return out

    def palmad_find_discords_resume(self, T, minL_sched: int, m0: int, maxL: int, topK: int, hist,
                                    options: Options | None = None, heatmap: bool = False) -> dict:
        """Lengths m0..maxL of a MERLIN run that started at minL_sched, from
        the schedule inputs of the lengths before m0 (see schedule_inputs)."""
        T = np.ascontiguousarray(T, dtype=np.float32)
        L = maxL - m0 + 1
        h = np.ascontiguousarray(hist, dtype=np.float64)
        idx = np.empty((L, topK), dtype=np.int64)
        nn = np.empty((L, topK), dtype=np.float64)
        cnt = np.empty(L, dtype=np.int64)
        rr = np.empty(L, dtype=np.float64)
        heat = np.empty((L, len(T) - m0 + 1), dtype=np.float32) if heatmap else None
        self._check(self._lib.palmad_find_discords_resume(
            self._h, _ptr(T), len(T), minL_sched, m0, maxL, topK, ctypes.byref(options) if options else None,
            _ptr(h) if len(h) else None, _ptr(idx), _ptr(nn), _ptr(cnt), _ptr(rr), _ptr(heat)))
        out = {"idx": idx, "nn": nn, "count": cnt, "r": rr}
        if heatmap:
            out["heatmap"] = heat
        return out

    def palmad_find_discords_device(self, T_dev, minL: int, maxL: int, topK: int,
                                    options: Options | None = None, heatmap_dev=None) -> dict:
        """Device-memory MERLIN: T_dev is a float32 CUDA tensor; outputs are
        CUDA tensors on the same device (allocated here through torch)."""
        import torch
        assert T_dev.is_cuda and T_dev.dtype == torch.float32 and T_dev.is_contiguous()
        L = maxL - minL + 1
        dev = T_dev.device
        idx = torch.empty((L, topK), dtype=torch.int64, device=dev)
        nn = torch.empty((L, topK), dtype=torch.float64, device=dev)
        cnt = torch.empty(L, dtype=torch.int64, device=dev)
        rr = torch.empty(L, dtype=torch.float64, device=dev)
        self._check(self._lib.palmad_find_discords_device(
            self._h, T_dev.data_ptr(), T_dev.numel(), minL, maxL, topK,
            ctypes.byref(options) if options else None, idx.data_ptr(), nn.data_ptr(), cnt.data_ptr(),
            rr.data_ptr(), heatmap_dev.data_ptr() if heatmap_dev is not None else None))
        return {"idx": idx, "nn": nn, "count": cnt, "r": rr}

    def palmad_autotune(self, T_dev, minL: int, maxL: int, topK: int, base: Options | None = None):
        """Tuned options for this series and length range (T_dev: float32
        CUDA tensor) and the tuner's report as a dict."""
        import torch
        assert T_dev.is_cuda and T_dev.dtype == torch.float32 and T_dev.is_contiguous()
        out = Options()
        rep = TuneReport()
        rep.struct_size = ctypes.sizeof(TuneReport)
        self._check(self._lib.palmad_autotune(self._h, T_dev.data_ptr(), T_dev.numel(), minL, maxL, topK,
                                              ctypes.byref(base) if base else None, ctypes.byref(out),
                                              ctypes.byref(rep)))
        report = {k: getattr(rep, k) for k, _ in rep._fields_ if k != "struct_size"}
        report["chosen"] = {k: getattr(out, k) for k in TUNED_FIELDS}
        return out, report

    def palmad_find_discords_batch(self, series, minL, maxL, topK: int, options: Options | None = None) -> list:
        """Independent series in one call; returns one result dict per series."""
        count = len(series)
        Ts = [np.ascontiguousarray(s, dtype=np.float32) for s in series]
        ns = np.array([len(s) for s in Ts], dtype=np.int64)
        mins = np.ascontiguousarray(minL, dtype=np.int32)
        maxs = np.ascontiguousarray(maxL, dtype=np.int32)
        outs = []
        for a, b in zip(mins, maxs):
            L = int(b) - int(a) + 1
            outs.append({"idx": np.empty((L, topK), dtype=np.int64), "nn": np.empty((L, topK)),
                         "count": np.empty(L, dtype=np.int64), "r": np.empty(L)})
        arr = lambda xs: (ctypes.c_void_p * count)(*[x.ctypes.data for x in xs])  # noqa: E731
        self._check(self._lib.palmad_find_discords_batch(
            self._h, count, arr(Ts), _ptr(ns), _ptr(mins), _ptr(maxs), topK,
            ctypes.byref(options) if options else None,
            arr([o["idx"] for o in outs]), arr([o["nn"] for o in outs]),
            arr([o["count"] for o in outs]), arr([o["r"] for o in outs])))
        return outs

    def palmad_drag_select_shard(self, T, m: int, r: float, row_lo: int, row_hi: int,
                                 options: Options | None = None) -> np.ndarray:
        """Candidate bitmap (uint32 words) of select over rows [row_lo, row_hi)."""
        T = np.ascontiguousarray(T, dtype=np.float32)
        bits = np.empty((len(T) - m + 1 + 31) // 32, dtype=np.uint32)
        self._check(self._lib.palmad_drag_select_shard(self._h, _ptr(T), len(T), m, float(r), row_lo, row_hi,
                                                       ctypes.byref(options) if options else None, _ptr(bits)))
        return bits

    def palmad_drag_refine_shard(self, T, m: int, r: float, cand_bits, col_lo: int, col_hi: int,
                                 options: Options | None = None) -> np.ndarray:
        """Per-window result of refining the candidates against columns
        [col_lo, col_hi): -1 pruned, else the FP64 distance over those columns."""
        T = np.ascontiguousarray(T, dtype=np.float32)
        bits = np.ascontiguousarray(cand_bits, dtype=np.uint32)
        out = np.empty(len(T) - m + 1, dtype=np.float64)
        self._check(self._lib.palmad_drag_refine_shard(self._h, _ptr(T), len(T), m, float(r), _ptr(bits), col_lo,
                                                       col_hi, ctypes.byref(options) if options else None, _ptr(out)))
        return out

    def palmad_drag(self, T, m: int, r: float, options: Options | None = None):
        """All range discords of length m at threshold r (ascending index)."""
        T = np.ascontiguousarray(T, dtype=np.float32)
        cap = 4096
        while True:
            idx = np.empty(cap, dtype=np.int64)
            nn = np.empty(cap, dtype=np.float64)
            cnt = ctypes.c_int64(0)
            self._check(self._lib.palmad_drag(self._h, _ptr(T), len(T), m, float(r),
                                              ctypes.byref(options) if options else None,
                                              _ptr(idx), _ptr(nn), cap, ctypes.byref(cnt)))
            if cnt.value <= cap:
                return idx[:cnt.value].copy(), nn[:cnt.value].copy()
            cap = cnt.value

"""GB300-native zSort: a stable distribution sort of (uint64 key, uint32 payload)
pairs after "zSort: Stable Distribution Sort using Z-Score Partitioning"
(arXiv 2605.14419).

This module is a thin ctypes binding of the C ABI in ``include/zsort.h``:
it only marshals arguments.  Every step of the sort runs in the CUDA library
``libzsort.so`` (built in-tree by ``paper_2605_14419_gb300.build``); there is
no CPU path.  PyTorch supplies device memory and streams only.

Tensors: keys are 8-byte CUDA tensors (torch.int64/uint64/float64 storage,
reinterpreted by ``key_type``), payloads 4-byte CUDA tensors (torch.int32 or
uint32 storage), both contiguous, sorted in place.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libzsort.so")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
_HEADERS = [os.path.join(_INCLUDE, h) for h in ("zsort.h", "zsort_tune.h")]
_lib = None

OK = 0
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_BAD_OFFSETS, ERR_CAPACITY, ERR_INTERNAL = (
    -1, -2, -3, -4, -5, -6, -7)
MAP_ZSCORE, MAP_LEARNED, MAP_MLP = 0, 1, 2
MAPINFO_ZSCORE, MAPINFO_LEARNED, MAPINFO_RANGE, MAPINFO_MLP, MAPINFO_SPLIT = 0, 1, 2, 3, 4
KEY_TYPES = {"u64": 0, "i64": 1, "f64": 2}
NOT_TUNED = 1
TUNE_FORCE = 1
TUNE_CLASS_MAX = 64
MAX_N = 1 << 30
MAX_SEG_TOTAL = 1 << 34
FLAG_GRAPH = 1
FLAG_TEST_STALL = 2
FLAG_TRACE = 4
FLAG_EXACT_SUBSTATS = 8
TILE_PAIRS = 3072  # at the default ipt (12 items per thread); 256 * ipt in general
SUB_SAMPLE = 4096
TRACE_CAP = 1 << 20
TASK_TYPES = {1: "stats", 2: "train", 3: "hist", 4: "scatter", 5: "mpart", 6: "finish", 7: "copy",
              8: "dump", 9: "fit", 10: "sampled stats"}
TRACE_HANDLER = 16
NOALLOC_MAX_N = 1 << 20


class ZsortError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class Opts(ctypes.Structure):
    """``zsort_opts`` (field meanings in include/zsort.h)."""

    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("mapper", ctypes.c_uint32),
        ("kmax", ctypes.c_uint32),
        ("leaf_target", ctypes.c_uint32),
        ("large_min", ctypes.c_uint32),
        ("learn_min", ctypes.c_uint32),
        ("sample", ctypes.c_uint32),
        ("fallback_ratio", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("guard_level", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32),
        ("wait_limit_ms", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("leaf_cap", ctypes.c_uint32),
        ("chunks_per_cta", ctypes.c_uint32),
        ("ipt", ctypes.c_uint32),
    ]


class Stats(ctypes.Structure):
    """``zsort_stats``: counters of the last call on a stream's workspace."""

    _fields_ = [
        ("n", ctypes.c_uint64),
        ("partitions_large", ctypes.c_uint64),
        ("partitions_small", ctypes.c_uint64),
        ("leaves", ctypes.c_uint64),
        ("leaf_fallbacks", ctypes.c_uint64),
        ("copies", ctypes.c_uint64),
        ("learned_accepted", ctypes.c_uint64),
        ("learned_rejected", ctypes.c_uint64),
        ("guard_levels", ctypes.c_uint64),
        ("max_level", ctypes.c_uint64),
        ("bytes_algorithmic", ctypes.c_uint64),
        ("tasks", ctypes.c_uint64),
        ("persistent_ctas", ctypes.c_uint64),
        ("top_mean_d", ctypes.c_double),
        ("top_sd", ctypes.c_double),
        ("top_min", ctypes.c_uint64),
        ("top_max", ctypes.c_uint64),
        ("top_k", ctypes.c_uint32),
        ("top_map", ctypes.c_uint32),
        ("task_ns", ctypes.c_uint64 * 8),
        ("task_count", ctypes.c_uint64 * 8),
        ("handler_ns", ctypes.c_uint64),
        ("idle_ns", ctypes.c_uint64),
        ("busy_window_ns", ctypes.c_uint64),
        ("sampled_stats", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class TraceRec(ctypes.Structure):
    """``zsort_trace_rec``: one task of the persistent kernel."""

    _fields_ = [
        ("t_start_ns", ctypes.c_uint64),
        ("t_end_ns", ctypes.c_uint64),
        ("cta", ctypes.c_uint32),
        ("type", ctypes.c_uint16),
        ("level", ctypes.c_uint16),
        ("arg", ctypes.c_uint32),
        ("count", ctypes.c_uint32),
    ]


class MapInfo(ctypes.Structure):
    """``zsort_map_info``: the top-level partition plan of one array."""

    _fields_ = [
        ("map", ctypes.c_uint32),
        ("k", ctypes.c_uint32),
        ("min", ctypes.c_uint64),
        ("max", ctypes.c_uint64),
        ("mean_d", ctypes.c_double),
        ("sd", ctypes.c_double),
        ("zc", ctypes.c_float),
        ("zsh", ctypes.c_uint32),
        ("escale", ctypes.c_float),
        ("trained", ctypes.c_uint32),
        ("q", ctypes.c_float * 257),
        ("r", ctypes.c_float * 256),
        ("learned_max_load", ctypes.c_uint32),
        ("zscore_max_load", ctypes.c_uint32),
        ("mlp", ctypes.c_float * 98),
    ]


def header_functions() -> list[str]:
    """Names of the functions declared in include/zsort.h and zsort_tune.h."""
    text = ""
    for h in _HEADERS:
        with open(h) as f:
            text += f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(zsort_\w+)\s*\(", text, re.M)))


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Loads libzsort.so; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"zsort CUDA library missing: {_LIB_PATH}; build it with "
                           "`python -m paper_2605_14419_gb300.build`")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "zsort_default_opts": (None, [ctypes.POINTER(Opts)]),
        "zsort_pairs": (i32, [vp, vp, u64, vp]),
        "zsort_keys": (i32, [vp, u64, vp]),
        "zsort_pairs_u128": (i32, [vp, vp, u64, ctypes.POINTER(Opts), vp]),
        "zsort_pairs_i64": (i32, [vp, vp, u64, vp]),
        "zsort_pairs_f64": (i32, [vp, vp, u64, vp]),
        "zsort_pairs_ex": (i32, [vp, u32, vp, u64, ctypes.POINTER(Opts), vp]),
        "zsort_segmented": (i32, [vp, vp, u64, vp, u64, vp]),
        "zsort_segmented_ex": (i32, [vp, vp, u64, vp, u64, ctypes.POINTER(Opts), vp]),
        "zsort_reserve": (i32, [u64, u64, vp]),
        "zsort_release": (i32, []),
        "zsort_sync_status": (i32, [vp]),
        "zsort_last_stats": (i32, [vp, ctypes.POINTER(Stats)]),
        "zsort_last_trace": (i32, [vp, ctypes.POINTER(TraceRec), u64, ctypes.POINTER(u64)]),
        "zsort_strerror": (ctypes.c_char_p, [i32]),
        "zsort_pairs_noalloc": (i32, [vp, vp, u64, vp, vp]),
        "zsort_map_buckets": (i32, [vp, u64, ctypes.POINTER(Opts), vp, ctypes.POINTER(MapInfo), vp]),
        "zsort_tune_class_host": (i32, [vp, u64, u64, u64, i32, ctypes.c_char_p, ctypes.c_size_t]),
        "zsort_tune_class": (i32, [vp, u64, u64, ctypes.c_char_p, ctypes.c_size_t, vp]),
        "zsort_tune_cache_get": (i32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Opts),
                                       ctypes.POINTER(ctypes.c_double)]),
        "zsort_tune_cache_put": (i32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Opts), ctypes.c_double]),
        "zsort_tuned_opts": (i32, [vp, u64, u64, ctypes.POINTER(Opts), ctypes.c_char_p, ctypes.POINTER(Opts), vp]),
        "zsort_autotune": (i32, [vp, vp, u64, vp, u64, ctypes.POINTER(Opts), ctypes.c_char_p, u32, u32, u32,
                                 ctypes.POINTER(Opts), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().zsort_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def default_opts(**overrides) -> Opts:
    o = Opts()
    load().zsort_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"zsort_opts has no field {k}")
        setattr(o, k, v)
    return o


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_tensor(t, elem: int, what: str):
    if not t.is_cuda or not t.is_contiguous() or t.element_size() != elem or t.dim() != 1:
        raise ValueError(f"{what}: need a contiguous 1-D CUDA tensor of {elem}-byte elements")


def _raise(rc: int, where: str):
    if rc != OK:
        raise ZsortError(rc, where)


def sort_pairs(keys, vals, key_type: str = "u64", opts: Opts | None = None, stream=None,
               check: bool = True):
    """Sorts (keys, vals) in place, stably by key; vals=None sorts the keys
    alone (key-only mode).  With check=True the stream is synchronised and
    the device status raised as ZsortError."""
    _check_tensor(keys, 8, "keys")
    if vals is not None:
        _check_tensor(vals, 4, "vals")
        if keys.numel() != vals.numel():
            raise ValueError("keys and vals differ in length")
    lib = load()
    st = _stream_handle(stream)
    rc = lib.zsort_pairs_ex(ctypes.c_void_p(keys.data_ptr()), KEY_TYPES[key_type],
                            ctypes.c_void_p(vals.data_ptr()) if vals is not None else None, keys.numel(),
                            ctypes.byref(opts) if opts is not None else None, st)
    _raise(rc, "zsort_pairs_ex")
    if check:
        _raise(lib.zsort_sync_status(st), "zsort (device)")
    return keys, vals


def sort_pairs_u128(keys, vals=None, opts: Opts | None = None, stream=None, check: bool = True):
    """Sorts 128-bit keys in place: keys is a contiguous CUDA int64 tensor of
    2n words (word 2i = low 64 bits of key i, 2i+1 = high); vals optional."""
    _check_tensor(keys, 8, "keys")
    if keys.numel() % 2:
        raise ValueError("keys: need 2 words per key")
    n = keys.numel() // 2
    if vals is not None:
        _check_tensor(vals, 4, "vals")
        if vals.numel() != n:
            raise ValueError("vals: need one payload per key")
    lib = load()
    st = _stream_handle(stream)
    rc = lib.zsort_pairs_u128(ctypes.c_void_p(keys.data_ptr()),
                              ctypes.c_void_p(vals.data_ptr()) if vals is not None else None, n,
                              ctypes.byref(opts) if opts is not None else None, st)
    _raise(rc, "zsort_pairs_u128")
    if check:
        _raise(lib.zsort_sync_status(st), "zsort_pairs_u128 (device)")
    return keys, vals


def sort_keys(keys, key_type: str = "u64", opts: Opts | None = None, stream=None, check: bool = True):
    """Key-only sort of keys in place."""
    return sort_pairs(keys, None, key_type=key_type, opts=opts, stream=stream, check=check)[0]


def sort_segmented(keys, vals, offsets, opts: Opts | None = None, stream=None, check: bool = True):
    """Sorts each segment [offsets[i], offsets[i+1]) of (keys, vals) in place
    (vals=None: keys only).  offsets: CUDA int64/uint64 tensor of nseg + 1
    entries."""
    _check_tensor(keys, 8, "keys")
    if vals is not None:
        _check_tensor(vals, 4, "vals")
    _check_tensor(offsets, 8, "offsets")
    lib = load()
    st = _stream_handle(stream)
    rc = lib.zsort_segmented_ex(ctypes.c_void_p(keys.data_ptr()),
                                ctypes.c_void_p(vals.data_ptr()) if vals is not None else None,
                                keys.numel(), ctypes.c_void_p(offsets.data_ptr()),
                                max(offsets.numel() - 1, 0),
                                ctypes.byref(opts) if opts is not None else None, st)
    _raise(rc, "zsort_segmented_ex")
    if check:
        _raise(lib.zsort_sync_status(st), "zsort_segmented (device)")
    return keys, vals


def map_buckets(keys, opts: Opts | None = None, stream=None):
    """Top-level bucket of every key (uint32 CUDA tensor) and the MapInfo."""
    import torch

    _check_tensor(keys, 8, "keys")
    out = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    info = MapInfo()
    rc = load().zsort_map_buckets(ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                  ctypes.byref(opts) if opts is not None else None,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.byref(info),
                                  _stream_handle(stream))
    _raise(rc, "zsort_map_buckets")
    return out, info


def reserve(n: int, nseg: int = 1, stream=None):
    _raise(load().zsort_reserve(n, nseg, _stream_handle(stream)), "zsort_reserve")


def release():
    _raise(load().zsort_release(), "zsort_release")


def sync_status(stream=None) -> int:
    return load().zsort_sync_status(_stream_handle(stream))


def last_stats(stream=None) -> dict:
    s = Stats()
    _raise(load().zsort_last_stats(_stream_handle(stream), ctypes.byref(s)), "zsort_last_stats")
    return s.as_dict()


def last_trace(stream=None, cap: int = TRACE_CAP):
    """Task trace of the last call on a stream (made with ``FLAG_TRACE``):
    (numpy structured array of the recorded tasks, number of tasks)."""
    import numpy as np

    buf = (TraceRec * max(cap, 1))()
    count = ctypes.c_uint64(0)
    _raise(load().zsort_last_trace(_stream_handle(stream), buf, cap, ctypes.byref(count)), "zsort_last_trace")
    m = min(count.value, cap, TRACE_CAP)
    dt = np.dtype([("t_start_ns", "<u8"), ("t_end_ns", "<u8"), ("cta", "<u4"), ("type", "<u2"),
                   ("level", "<u2"), ("arg", "<u4"), ("count", "<u4")])
    assert dt.itemsize == ctypes.sizeof(TraceRec)
    arr = np.frombuffer(ctypes.string_at(ctypes.addressof(buf), m * dt.itemsize), dtype=dt).copy()
    return arr, count.value


# ------------------------------------------------------------ autotuner
def _path(p):
    return None if p is None else os.fsencode(p)


def tune_class_host(sample, n: int, nseg: int = 0, sms: int = 152) -> str:
    """Class string of a call from a host sample (numpy uint64 array)."""
    import numpy as np

    a = np.ascontiguousarray(sample, dtype=np.uint64)
    buf = ctypes.create_string_buffer(TUNE_CLASS_MAX)
    _raise(load().zsort_tune_class_host(a.ctypes.data if a.size else None, a.size, n, nseg, sms, buf,
                                        TUNE_CLASS_MAX), "zsort_tune_class_host")
    return buf.value.decode()


def tune_class(keys, nseg: int = 0, stream=None) -> str:
    _check_tensor(keys, 8, "keys")
    buf = ctypes.create_string_buffer(TUNE_CLASS_MAX)
    _raise(load().zsort_tune_class(ctypes.c_void_p(keys.data_ptr()), keys.numel(), nseg, buf, TUNE_CLASS_MAX,
                                   _stream_handle(stream)), "zsort_tune_class")
    return buf.value.decode()


def tune_cache_get(path: str, cls: str, base: Opts | None = None):
    """(Opts, ms) of a cache entry, or None if the class is not cached."""
    o = base if base is not None else default_opts()
    o = Opts.from_buffer_copy(o)
    ms = ctypes.c_double(0.0)
    rc = load().zsort_tune_cache_get(_path(path), cls.encode(), ctypes.byref(o), ctypes.byref(ms))
    if rc == NOT_TUNED:
        return None
    _raise(rc, "zsort_tune_cache_get")
    return o, ms.value


def tune_cache_put(path: str, cls: str, opts: Opts, ms: float):
    _raise(load().zsort_tune_cache_put(_path(path), cls.encode(), ctypes.byref(opts), ms), "zsort_tune_cache_put")


def tuned_opts(keys, nseg: int = 0, base: Opts | None = None, cache_path: str | None = None, stream=None):
    """(Opts, found): the base options with the cached tuned fields of the call's class."""
    _check_tensor(keys, 8, "keys")
    out = Opts()
    rc = load().zsort_tuned_opts(ctypes.c_void_p(keys.data_ptr()), keys.numel(), nseg,
                                 ctypes.byref(base) if base is not None else None, _path(cache_path),
                                 ctypes.byref(out), _stream_handle(stream))
    if rc not in (OK, NOT_TUNED):
        _raise(rc, "zsort_tuned_opts")
    return out, rc == OK


def autotune(keys, vals, offsets=None, base: Opts | None = None, cache_path: str | None = None,
             budget_ms: int = 0, reps: int = 3, force: bool = False, stream=None) -> Opts:
    """Tuned options for sorting (keys, vals) -- or the segmented batch when
    offsets is given; the tensors are not modified."""
    _check_tensor(keys, 8, "keys")
    _check_tensor(vals, 4, "vals")
    if offsets is not None:
        _check_tensor(offsets, 8, "offsets")
    out = Opts()
    rc = load().zsort_autotune(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()), keys.numel(),
                               ctypes.c_void_p(offsets.data_ptr()) if offsets is not None else None,
                               max(offsets.numel() - 1, 0) if offsets is not None else 0,
                               ctypes.byref(base) if base is not None else None, _path(cache_path), budget_ms, reps,
                               TUNE_FORCE if force else 0, ctypes.byref(out), _stream_handle(stream))
    _raise(rc, "zsort_autotune")
    return out

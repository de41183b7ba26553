"""CPU oracle for zSort: a plain, sequential C restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg (``bench.py --impl reference`` and the
``cpu_baseline`` object) may import this package.  The product library never
does, and the two share no code: see ``zsort_oracle.c`` for the citations.

The C file is compiled with plain ``gcc -O2`` (no fast-math, no FP
contraction), and ``baseline_cpu.cpp`` (std::stable_sort and a std::thread
pool over segments, the CPU comparison sorts of the benchmark) with ``g++
-O2``, into ``oracle/liboracle.so`` on first use, or by ``build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zsort_oracle.c")
_SRC_CPP = os.path.join(_HERE, "baseline_cpu.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

P_PIECES = 256  # breakpoints of the learned map: q[0..P]


class Trace(ctypes.Structure):
    """Counters of one oracle run (mirrors ``oracle_trace`` in the C file)."""

    _fields_ = [
        ("partitions", ctypes.c_uint64),
        ("max_depth", ctypes.c_uint64),
        ("guard_levels", ctypes.c_uint64),
        ("counting_sorts", ctypes.c_uint64),
        ("insertion_sorts", ctypes.c_uint64),
        ("equal_exits", ctypes.c_uint64),
        ("k", ctypes.c_uint64),
        ("scale", ctypes.c_double),
    ]


class SubRec(ctypes.Structure):
    """One zsortRec sub-problem (mirrors ``oracle_sub_rec`` in the C file)."""

    _fields_ = [
        ("depth", ctypes.c_uint64),
        ("parent_bucket", ctypes.c_uint64),
        ("size", ctypes.c_uint64),
        ("min", ctypes.c_uint64),
        ("parent_min", ctypes.c_uint64),
        ("est_parent_d", ctypes.c_double),
        ("mean", ctypes.c_double),
        ("sd", ctypes.c_double),
        ("zmin", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc/g++; returns the path of the shared library."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_CPP))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
            tag = f".tmp{os.getpid()}"
            obj_c, obj_cpp, tmp = _LIB + tag + ".c.o", _LIB + tag + ".cpp.o", _LIB + tag
            try:
                subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-c",
                                "-o", obj_c, _SRC], check=True)
                subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-c", "-o", obj_cpp, _SRC_CPP], check=True)
                subprocess.run(["g++", "-shared", "-o", tmp, obj_c, obj_cpp, "-lm", "-pthread"], check=True)
                os.replace(tmp, _LIB)
            finally:
                for f in (obj_c, obj_cpp):
                    if os.path.exists(f):
                        os.remove(f)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_zsort_pairs_ex.restype = ctypes.c_int
        lib.oracle_zsort_pairs_ex.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                              ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_uint64, ctypes.POINTER(Trace)]
        lib.oracle_zsort_pairs_rec.restype = ctypes.c_int
        lib.oracle_zsort_pairs_rec.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                               ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.POINTER(Trace),
                                               ctypes.POINTER(SubRec), ctypes.c_uint64, u64p]
        lib.oracle_zsort_segmented.restype = ctypes.c_int
        lib.oracle_zsort_segmented.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_uint64]
        lib.oracle_stdsort_pairs.restype = ctypes.c_int
        lib.oracle_stdsort_pairs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
        lib.oracle_zsort_segmented_mt.restype = ctypes.c_int
        lib.oracle_zsort_segmented_mt.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_uint64, ctypes.c_int]
        lib.oracle_stats.restype = None
        lib.oracle_stats.argtypes = [ctypes.c_void_p, ctypes.c_uint64, u64p, u64p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        for name in ("oracle_key_from_i64", "oracle_key_to_i64", "oracle_key_from_f64",
                     "oracle_key_to_f64"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
        lib.oracle_level1_buckets.restype = None
        lib.oracle_level1_buckets.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_void_p]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        lib.oracle_sample_positions.restype = None
        lib.oracle_sample_positions.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                                ctypes.c_void_p]
        lib.oracle_pwl_normalise.restype = ctypes.c_float
        lib.oracle_pwl_normalise.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_pwl_train.restype = None
        lib.oracle_pwl_train.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_pwl_buckets.restype = None
        lib.oracle_pwl_buckets.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_pwl_bucket.restype = ctypes.c_uint32
        lib.oracle_pwl_bucket.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_split_train.restype = None
        lib.oracle_split_train.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_split_buckets.restype = None
        lib.oracle_split_buckets.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_mlp_train.restype = None
        lib.oracle_mlp_train.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_mlp_buckets.restype = None
        lib.oracle_mlp_buckets.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_mlp_eval.restype = ctypes.c_float
        lib.oracle_mlp_eval.argtypes = [ctypes.c_void_p, ctypes.c_float]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def zsort_pairs(keys, vals, alpha: float = 0.6, leaf: int = 96, count_range: int = 65000,
                guard_depth: int = 32, with_trace: bool = False):
    """Paper's zSort (Alg. 1 + zsortRec) on (uint64 key, uint32 payload) pairs.

    Returns sorted copies (keys, vals) and, if asked, the run's Trace.
    """
    k = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    assert k.shape == v.shape and k.ndim == 1
    tr = Trace()
    rc = _load().oracle_zsort_pairs_ex(_ptr(k), _ptr(v), k.size, alpha, leaf, count_range,
                                       guard_depth, ctypes.byref(tr))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (k, v, tr) if with_trace else (k, v)


def zsort_pairs_records(keys, vals, alpha: float = 0.6, leaf: int = 96, count_range: int = 65000,
                        guard_depth: int = 32, cap: int = 1 << 16):
    """As zsort_pairs, and the list of zsortRec sub-problems (SubRec) the run
    partitioned, in the order it visited them (R9: meanEst, mean, sd, Zmin)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    tr = Trace()
    recs = (SubRec * cap)()
    cnt = ctypes.c_uint64()
    rc = _load().oracle_zsort_pairs_rec(_ptr(k), _ptr(v), k.size, alpha, leaf, count_range, guard_depth,
                                        ctypes.byref(tr), recs, cap, ctypes.byref(cnt))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return k, v, tr, [recs[i] for i in range(min(cnt.value, cap))]


def zsort_segmented(keys, vals, offsets):
    """Each segment [offsets[i], offsets[i+1]) sorted on its own (copies)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = _load().oracle_zsort_segmented(_ptr(k), _ptr(v), _ptr(off), off.size - 1)
    if rc != 0:
        raise ValueError(f"oracle_zsort_segmented failed: {rc}")
    return k, v


def stdsort_pairs(keys, vals):
    """std::stable_sort of the pairs by key, one thread (a comparison sort)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    _load().oracle_stdsort_pairs(_ptr(k), _ptr(v), k.size)
    return k, v


def zsort_segmented_mt(keys, vals, offsets, threads: int = 0):
    """The oracle's zSort of every segment, segments shared out over a pool
    of `threads` host threads (0: one per core).  Returns (keys, vals,
    threads used)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    t = _load().oracle_zsort_segmented_mt(_ptr(k), _ptr(v), _ptr(off), off.size - 1, threads)
    if t < 0:
        raise ValueError(f"oracle_zsort_segmented_mt failed: {t}")
    return k, v, t


def stats(keys):
    """(min, max, mean of key-min, population sd) as in Alg. 1's first loops."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    mn, mx = ctypes.c_uint64(), ctypes.c_uint64()
    mean, sd = ctypes.c_double(), ctypes.c_double()
    _load().oracle_stats(_ptr(k), k.size, ctypes.byref(mn), ctypes.byref(mx),
                         ctypes.byref(mean), ctypes.byref(sd))
    return mn.value, mx.value, mean.value, sd.value


def level1_buckets(keys, k: int):
    """Cluster index of every key under Eq. 1 at the top level."""
    a = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(a.size, dtype=np.uint64)
    _load().oracle_level1_buckets(_ptr(a), a.size, k, _ptr(out))
    return out


def key_from_i64(x):
    a = np.ascontiguousarray(x, dtype=np.int64)
    out = np.empty(a.size, dtype=np.uint64)
    _load().oracle_key_from_i64(_ptr(a), _ptr(out), a.size)
    return out


def key_to_i64(u):
    a = np.ascontiguousarray(u, dtype=np.uint64)
    out = np.empty(a.size, dtype=np.int64)
    _load().oracle_key_to_i64(_ptr(a), _ptr(out), a.size)
    return out


def key_from_f64(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(a.size, dtype=np.uint64)
    _load().oracle_key_from_f64(_ptr(a), _ptr(out), a.size)
    return out


def key_to_f64(u):
    a = np.ascontiguousarray(u, dtype=np.uint64)
    out = np.empty(a.size, dtype=np.float64)
    _load().oracle_key_to_f64(_ptr(a), _ptr(out), a.size)
    return out


def splitmix64(x: int) -> int:
    return int(_load().oracle_splitmix64(x))


def sample_positions(seed: int, length: int, m: int):
    pos = np.empty(m, dtype=np.uint64)
    _load().oracle_sample_positions(seed, length, m, _ptr(pos))
    return pos


def pwl_normalise(key: int, mn: int, mx: int) -> float:
    return float(_load().oracle_pwl_normalise(key, mn, mx))


def pwl_train(sample_keys, mn: int, mx: int, P: int = P_PIECES):
    s = np.ascontiguousarray(sample_keys, dtype=np.uint64)
    q = np.empty(P + 1, dtype=np.float32)
    _load().oracle_pwl_train(_ptr(s), s.size, mn, mx, P, _ptr(q))
    return q


def pwl_buckets(keys, mn: int, mx: int, q, k: int, P: int = P_PIECES):
    """Learned-map bucket of every key."""
    qq = np.ascontiguousarray(q, dtype=np.float32)
    kk = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(kk.size, dtype=np.uint32)
    _load().oracle_pwl_buckets(_ptr(kk), kk.size, mn, mx, _ptr(qq), P, k, _ptr(out))
    return out


def learned_map(keys, seed: int, m: int, k: int, P: int = P_PIECES):
    """Whole learned-mapper training step on one array: the sample drawn at
    splitmix64-stratified positions, the exact min/max of the array, the
    breakpoints, and the map's bucket of every sample key."""
    k_arr = np.ascontiguousarray(keys, dtype=np.uint64)
    mn, mx = int(k_arr.min()), int(k_arr.max())
    pos = sample_positions(seed, k_arr.size, m)
    sample = k_arr[pos.astype(np.int64)]
    q = pwl_train(sample, mn, mx, P)
    return mn, mx, q, sample


def split_train(sample_keys, mn: int, mx: int, P: int = P_PIECES):
    """Exact-key breakpoints b[0..P] (uint64) and stored slopes r[0..P) of the
    learned map's second form."""
    srt = np.ascontiguousarray(sample_keys, dtype=np.uint64)
    b = np.empty(P + 1, dtype=np.uint64)
    r = np.empty(P, dtype=np.float32)
    _load().oracle_split_train(_ptr(srt), srt.size, mn, mx, P, _ptr(b), _ptr(r))
    return b, r


def split_buckets(keys, b, r, k: int, P: int = P_PIECES):
    kk = np.ascontiguousarray(keys, dtype=np.uint64)
    bb = np.ascontiguousarray(b, dtype=np.uint64)
    rr = np.ascontiguousarray(r, dtype=np.float32)
    out = np.empty(kk.size, dtype=np.uint32)
    _load().oracle_split_buckets(_ptr(kk), kk.size, _ptr(bb), _ptr(rr), P, k, _ptr(out))
    return out


MLP_H = 32
MLP_PARAMS = 3 * MLP_H + 2


def mlp_train(q, iters: int):
    """Trained MLP map parameters (omega, beta, alpha, f0, inv) from the knots q."""
    qq = np.ascontiguousarray(q, dtype=np.float32)
    out = np.empty(MLP_PARAMS, dtype=np.float32)
    _load().oracle_mlp_train(_ptr(qq), qq.size - 1, iters, _ptr(out))
    return out


def mlp_buckets(keys, mn: int, mx: int, params, k: int):
    kk = np.ascontiguousarray(keys, dtype=np.uint64)
    pp = np.ascontiguousarray(params, dtype=np.float32)
    out = np.empty(kk.size, dtype=np.uint32)
    _load().oracle_mlp_buckets(_ptr(kk), kk.size, mn, mx, _ptr(pp), k, _ptr(out))
    return out


def mlp_eval(params, u: float) -> float:
    pp = np.ascontiguousarray(params, dtype=np.float32)
    return float(_load().oracle_mlp_eval(_ptr(pp), ctypes.c_float(u)))

"""CPU oracle for the hybrid Quicksort hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (``bench.py --impl reference`` and the ``cpu_baseline`` field) may import
this package.  The product path (``paper_1704_08579_gb300``) never does and
shares no code with it.

The arithmetic lives in ``qs_oracle.cpp`` (plain C++, no library algorithms);
this module compiles it with the host compiler and wraps it with ctypes.
What each function follows in the paper is stated in the C++ file's header:
partition = Section III-B with a fixed (input-order / reverse-input-order)
arrangement, sort = Appendix A scalar Quicksort, key/value = Section III-D.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle shared library (portable C++, no ISA-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.oracle_partition_i32.argtypes = [vp, vp, i64, i32]
            lib.oracle_partition_i32.restype = i64
            lib.oracle_partition_f64.argtypes = [vp, vp, i64, f64]
            lib.oracle_partition_f64.restype = i64
            lib.oracle_partition_kv.argtypes = [vp, vp, vp, vp, i64, i32]
            lib.oracle_partition_kv.restype = i64
            lib.oracle_sort_i32.argtypes = [vp, i64]
            lib.oracle_sort_i32.restype = ctypes.c_int
            lib.oracle_sort_f64.argtypes = [vp, i64]
            lib.oracle_sort_f64.restype = ctypes.c_int
            lib.oracle_sort_kv.argtypes = [vp, vp, i64]
            lib.oracle_sort_kv.restype = ctypes.c_int
            for name in ("oracle_sort_par_i32", "oracle_sort_par_f64"):
                getattr(lib, name).argtypes = [vp, i64, ctypes.c_int]
                getattr(lib, name).restype = ctypes.c_int
            lib.oracle_sort_par_kv.argtypes = [vp, vp, i64, ctypes.c_int]
            lib.oracle_sort_par_kv.restype = ctypes.c_int
            lib.oracle_sort_trace_i32.argtypes = [vp, i64, vp, i64, vp]
            lib.oracle_sort_trace_i32.restype = ctypes.c_int
            lib.oracle_select_i32.argtypes = [vp, i64, i64]
            lib.oracle_select_i32.restype = i32
            lib.oracle_select_f64.argtypes = [vp, i64, i64]
            lib.oracle_select_f64.restype = f64
            lib.oracle_mlp_nparams.argtypes = []
            lib.oracle_mlp_nparams.restype = ctypes.c_long
            lib.oracle_mlp_forward.argtypes = [vp, vp, ctypes.c_long, vp]
            lib.oracle_mlp_forward.restype = None
            lib.oracle_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_long, vp]
            lib.oracle_mlp_loss_grad.restype = f64
            lib.oracle_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_long, ctypes.c_long, f64, f64, f64, f64]
            lib.oracle_adam_step.restype = None
            for name in ("oracle_bucket_i32", "oracle_bucket_f64"):
                fn = getattr(lib, name)
                fn.argtypes = [vp, vp, ctypes.c_long, vp, ctypes.c_int, vp]
                fn.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def partition(keys: np.ndarray, pivot, values: np.ndarray | None = None):
    """Out-of-place partition.  Returns (split, keys_out[, values_out])."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    n = keys.size
    if values is not None:
        values = np.ascontiguousarray(values, dtype=np.int32)
        vout = np.empty_like(values)
        split = lib.oracle_partition_kv(_p(keys), _p(values), _p(out), _p(vout), n, int(pivot))
        return split, out, vout
    if keys.dtype == np.int32:
        split = lib.oracle_partition_i32(_p(keys), _p(out), n, int(pivot))
    elif keys.dtype == np.float64:
        split = lib.oracle_partition_f64(_p(keys), _p(out), n, float(pivot))
    else:
        raise TypeError(keys.dtype)
    return split, out


def sort(keys: np.ndarray, values: np.ndarray | None = None):
    """Returns sorted copies: keys, or (keys, values) for key/value input."""
    lib = _load()
    k = np.array(keys, copy=True, order="C")
    if values is not None:
        v = np.array(values, dtype=np.int32, copy=True, order="C")
        rc = lib.oracle_sort_kv(_p(k), _p(v), k.size)
        if rc:
            raise MemoryError("oracle stack")
        return k, v
    if k.dtype == np.int32:
        rc = lib.oracle_sort_i32(_p(k), k.size)
    elif k.dtype == np.float64:
        rc = lib.oracle_sort_f64(_p(k), k.size)
    else:
        raise TypeError(k.dtype)
    if rc:
        raise MemoryError("oracle stack")
    return k


def sort_parallel(keys: np.ndarray, values: np.ndarray | None = None, threads: int | None = None):
    """Sorted copies like sort(), computed by the task-parallel oracle (same result bit for bit)."""
    lib = _load()
    t = threads or os.cpu_count() or 1
    k = np.array(keys, copy=True, order="C")
    if values is not None:
        v = np.array(values, dtype=np.int32, copy=True, order="C")
        if lib.oracle_sort_par_kv(_p(k), _p(v), k.size, t):
            raise MemoryError("oracle stack")
        return k, v
    fn = lib.oracle_sort_par_i32 if k.dtype == np.int32 else lib.oracle_sort_par_f64
    if k.dtype not in (np.int32, np.float64):
        raise TypeError(k.dtype)
    if fn(_p(k), k.size, t):
        raise MemoryError("oracle stack")
    return k


def sort_inplace(keys: np.ndarray) -> None:
    """In-place sort of a contiguous int32/float64 array (used for timing the baseline)."""
    lib = _load()
    fn = lib.oracle_sort_i32 if keys.dtype == np.int32 else lib.oracle_sort_f64
    if fn(_p(keys), keys.size):
        raise MemoryError("oracle stack")


def sort_trace(keys: np.ndarray, cap: int = 1 << 16):
    """Sorted copy of int32 keys plus the pivots in the order Appendix A picks them."""
    lib = _load()
    k = np.array(keys, dtype=np.int32, copy=True)
    trace = np.zeros(cap, dtype=np.float64)
    nt = ctypes.c_int64(0)
    rc = lib.oracle_sort_trace_i32(_p(k), k.size, _p(trace), cap, ctypes.byref(nt))
    if rc:
        raise MemoryError("oracle stack")
    return k, trace[: min(nt.value, cap)]


def select(keys: np.ndarray, k: int):
    """k-th smallest (0-based) key."""
    lib = _load()
    a = np.array(keys, copy=True, order="C")
    if a.dtype == np.int32:
        return int(lib.oracle_select_i32(_p(a), a.size, int(k)))
    if a.dtype == np.float64:
        return float(lib.oracle_select_f64(_p(a), a.size, int(k)))
    raise TypeError(a.dtype)


# ---------------------------------------------------------------------------
# Learned-splitter growth line: MLP in double precision and bucket partition.
# ---------------------------------------------------------------------------
MLP_IN, MLP_HID, MLP_OUT, MLP_SPLIT = 1024, 64, 256, 255


def mlp_nparams() -> int:
    return int(_load().oracle_mlp_nparams())


def mlp_forward(params: np.ndarray, x: np.ndarray) -> np.ndarray:
    """q (batch x 255) for sketches x (batch x 1024)."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    q = np.empty((xx.shape[0], MLP_SPLIT), dtype=np.float64)
    lib.oracle_mlp_forward(_p(p), _p(xx), xx.shape[0], _p(q))
    return q


def mlp_loss_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(loss, gradient) of the mean squared quantile error."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    tt = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, MLP_SPLIT)
    g = np.empty_like(p)
    loss = lib.oracle_mlp_loss_grad(_p(p), _p(xx), _p(tt), xx.shape[0], _p(g))
    return float(loss), g


def bucket(keys: np.ndarray, splitters: np.ndarray):
    """Stable bucket partition: (out, counts) with bucket(k) = #splitters <= k."""
    lib = _load()
    k = np.ascontiguousarray(keys)
    s = np.ascontiguousarray(splitters, dtype=k.dtype)
    out = np.empty_like(k)
    counts = np.empty(s.size + 1, dtype=np.int64)
    fn = lib.oracle_bucket_i32 if k.dtype == np.int32 else lib.oracle_bucket_f64
    fn(_p(k), _p(out), k.size, _p(s), s.size, _p(counts))
    return out, counts


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on copies; returns (p, m, v)."""
    lib = _load()
    p = np.array(p, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib.oracle_adam_step(_p(p), _p(g), _p(m), _p(v), p.size, int(step), lr, b1, b2, eps)
    return p, m, v

"""Python binding of libqs.so, the GB300 (sm_103a) hybrid Quicksort library.

Argument marshalling only: every step of partitioning and sorting runs in the
library's CUDA kernels.  The names follow the C-ABI in ``include/qs.h``:

    partition(keys, pivot, values=None)  -> split index   (qs_partition_*)
    sort(keys, values=None, sync=True)                    (qs_sort_*)
    sort_host(keys, values=None)                          (qs_sort_host_*)
    sync_status(stream=None)                              (qs_sync_status)

The C sorts are asynchronous; ``sort``/``sort_segmented`` call
``qs_sync_status`` after them (raising on a device-side failure) unless
``sync=False`` is passed, in which case a failure is raised by a later
``sync_status`` or by the next call.

``keys``/``values`` are contiguous CUDA tensors (int32 or float64 keys, int32
values) for ``partition``/``sort`` and contiguous numpy arrays for
``sort_host``.  Work is issued on the current torch CUDA stream (or the one
passed).  There is no CPU fallback: if the library has not been built, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libqs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "qs.h")

QS_OK = 0
STATUS = {
    -1: "QS_ERR_INVALID_ARG", -2: "QS_ERR_ALIGN", -3: "QS_ERR_OOM", -4: "QS_ERR_CUDA",
    -5: "QS_ERR_TIMEOUT", -6: "QS_ERR_CAPACITY", -7: "QS_ERR_INTERNAL",
}
KIND = {"i32": 0, "f64": 1, "kv": 2}
OPTION = {"profile": 1, "wait_limit_ns": 2, "task_cap": 3, "driver_ctas": 4, "leaf_max": 5, "small_max": 6,
          "driver_items": 7, "ordered": 8, "sync": 9, "bucket_levels": 10}

_lib = None
_lock = threading.Lock()


class QSError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "QS_ERR"), code, message))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n", "kind", "part_tasks", "part_keys", "leaf_parts", "leaf_keys", "copy_keys", "max_depth",
        "lookback_words", "grid_driver", "grid_leaf")] + [
        (name, ctypes.c_double) for name in ("ms_driver", "ms_leaf", "ms_copy", "ms_total")] + [
        ("driver_cycles", ctypes.c_int64 * 40), ("bucket_max", ctypes.c_int64), ("bucket_over", ctypes.c_int64),
        ("bucket_dev", ctypes.c_int64), ("mid_parts", ctypes.c_int64), ("mid_keys", ctypes.c_int64)]


def header_functions() -> list[str]:
    """Names of the functions declared in include/qs.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    """Loads libqs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqs.so is not built (%s); run paper_1704_08579_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        i64, i32, f64, vp, ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
        sig = {
            "qs_partition_i32": ([vp, i64, i32, vp], i64),
            "qs_partition_f64": ([vp, i64, f64, vp], i64),
            "qs_partition_kv": ([vp, vp, i64, i32, vp], i64),
            "qs_partition_i32_noalloc": ([vp, i64, i32, vp], i64),
            "qs_sort_i32": ([vp, i64, vp], ci),
            "qs_sort_f64": ([vp, i64, vp], ci),
            "qs_sort_kv": ([vp, vp, i64, vp], ci),
            "qs_sort_segmented_i32": ([vp, i64, vp, i64, vp], ci),
            "qs_sort_segmented_f64": ([vp, i64, vp, i64, vp], ci),
            "qs_sort_segmented_kv": ([vp, vp, i64, vp, i64, vp], ci),
            "qs_sort_learned_i32": ([vp, i64, vp, vp], ci),
            "qs_sort_learned_f64": ([vp, i64, vp, vp], ci),
            "qs_bucket_i32": ([vp, i64, vp, ci, vp, vp], ci),
            "qs_bucket_f64": ([vp, i64, vp, ci, vp, vp], ci),
            "qs_sketch_i32": ([vp, i64, vp, vp, vp, vp], ci),
            "qs_sketch_f64": ([vp, i64, vp, vp, vp, vp], ci),
            "qs_mlp_param_count": ([], ci),
            "qs_mlp_forward": ([vp, vp, i64, vp, vp, vp], ci),
            "qs_mlp_backward": ([vp, vp, vp, vp, i64, vp, vp, vp, vp], ci),
            "qs_mlp_adam": ([vp, vp, vp, vp, i64, ctypes.c_float, vp], ci),
            "qs_sort_host_i32": ([vp, i64, vp], ci),
            "qs_sort_host_f64": ([vp, i64, vp], ci),
            "qs_sort_host_kv": ([vp, vp, i64, vp], ci),
            "qs_sync_status": ([vp], ci),
            "qs_reserve": ([i64, ci], ci),
            "qs_release": ([], None),
            "qs_last_error": ([], ctypes.c_char_p),
            "qs_version": ([], ci),
            "qs_get_stats": ([ctypes.POINTER(Stats)], ci),
            "qs_set_option": ([ci, i64], ci),
            "qs_get_option": ([ci, ctypes.POINTER(i64)], ci),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load().qs_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise QSError(rc, last_error())
    return rc


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _kind_of(keys, values) -> str:
    import torch

    if values is not None:
        if keys.dtype != torch.int32 or values.dtype != torch.int32:
            raise TypeError("key/value sorting takes int32 keys and int32 values")
        return "kv"
    if keys.dtype == torch.int32:
        return "i32"
    if keys.dtype == torch.float64:
        return "f64"
    raise TypeError("keys must be int32 or float64, got %s" % keys.dtype)


def _check_tensor(t, name):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def partition(keys, pivot, values=None, stream=None) -> int:
    """qs_partition_*: reorders keys (and values) around pivot; returns the split index."""
    lib = load()
    kind = _kind_of(keys, values)
    _check_tensor(keys, "keys")
    s = _stream_handle(stream)
    n = keys.numel()
    if kind == "kv":
        _check_tensor(values, "values")
        if values.numel() != n:
            raise ValueError("keys and values differ in length")
        return _check(lib.qs_partition_kv(keys.data_ptr(), values.data_ptr(), n, int(pivot), s))
    if kind == "i32":
        return _check(lib.qs_partition_i32(keys.data_ptr(), n, int(pivot), s))
    return _check(lib.qs_partition_f64(keys.data_ptr(), n, float(pivot), s))


def sync_status(stream=None) -> None:
    """qs_sync_status: waits for the library's work and for `stream`; raises
    the first device-side failure of an asynchronous call not reported yet."""
    _check(load().qs_sync_status(_stream_handle(stream)))


def sort(keys, values=None, stream=None, sync=True) -> None:
    """qs_sort_*: sorts keys (and values with them) in place; with
    sync=False it returns once the work is enqueued."""
    lib = load()
    kind = _kind_of(keys, values)
    _check_tensor(keys, "keys")
    s = _stream_handle(stream)
    n = keys.numel()
    if kind == "kv":
        _check_tensor(values, "values")
        if values.numel() != n:
            raise ValueError("keys and values differ in length")
        _check(lib.qs_sort_kv(keys.data_ptr(), values.data_ptr(), n, s))
    elif kind == "i32":
        _check(lib.qs_sort_i32(keys.data_ptr(), n, s))
    else:
        _check(lib.qs_sort_f64(keys.data_ptr(), n, s))
    if sync:
        _check(lib.qs_sync_status(s))


def sort_segmented(keys, offsets, values=None, stream=None, sync=True) -> None:
    """qs_sort_segmented_*: sorts every segment [offsets[i], offsets[i+1]) of keys in place.

    ``offsets`` is a CUDA int64 tensor of nseg + 1 entries."""
    import torch

    lib = load()
    kind = _kind_of(keys, values)
    _check_tensor(keys, "keys")
    _check_tensor(offsets, "offsets")
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    s = _stream_handle(stream)
    n = keys.numel()
    nseg = max(offsets.numel() - 1, 0)
    if kind == "kv":
        _check_tensor(values, "values")
        if values.numel() != n:
            raise ValueError("keys and values differ in length")
        _check(lib.qs_sort_segmented_kv(keys.data_ptr(), values.data_ptr(), n, offsets.data_ptr(), nseg, s))
    elif kind == "i32":
        _check(lib.qs_sort_segmented_i32(keys.data_ptr(), n, offsets.data_ptr(), nseg, s))
    else:
        _check(lib.qs_sort_segmented_f64(keys.data_ptr(), n, offsets.data_ptr(), nseg, s))
    if sync:
        _check(lib.qs_sync_status(s))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def sort_learned(keys, params=None, stream=None) -> None:
    """qs_sort_learned_*: 256-way bucket pass by learned (params) or sampled
    (params=None) splitters, then the plain method in every bucket."""
    import torch

    lib = load()
    _check_tensor(keys, "keys")
    s = _stream_handle(stream)
    if params is not None:
        _check_tensor(params, "params")
        if params.dtype != torch.float32 or params.numel() != lib.qs_mlp_param_count():
            raise ValueError("params must be %d float32 values" % lib.qs_mlp_param_count())
    fn = {torch.int32: lib.qs_sort_learned_i32, torch.float64: lib.qs_sort_learned_f64}.get(keys.dtype)
    if fn is None:
        raise TypeError("learned sort takes int32 or float64 keys")
    _check(fn(keys.data_ptr(), keys.numel(), _ptr(params), s))


def bucket(keys, splitters, stream=None):
    """qs_bucket_*: groups keys into nsplit + 1 buckets in place; returns the
    int64 CUDA tensor of bucket starts (nsplit + 2 entries, last = n)."""
    import torch

    lib = load()
    _check_tensor(keys, "keys")
    _check_tensor(splitters, "splitters")
    if splitters.dtype != keys.dtype:
        raise TypeError("splitters must have the keys' dtype")
    off = torch.empty(splitters.numel() + 2, dtype=torch.int64, device=keys.device)
    fn = {torch.int32: lib.qs_bucket_i32, torch.float64: lib.qs_bucket_f64}.get(keys.dtype)
    if fn is None:
        raise TypeError("bucket pass takes int32 or float64 keys")
    _check(fn(keys.data_ptr(), keys.numel(), splitters.data_ptr(), splitters.numel(), off.data_ptr(),
              _stream_handle(stream)))
    return off


def sketch(keys, stream=None):
    """qs_sketch_*: (sketch float32[1024], minmax float64[2], sorted sample keys[1024]) CUDA tensors."""
    import torch

    lib = load()
    _check_tensor(keys, "keys")
    x = torch.empty(1024, dtype=torch.float32, device=keys.device)
    mm = torch.empty(2, dtype=torch.float64, device=keys.device)
    smp = torch.empty(1024, dtype=keys.dtype, device=keys.device)
    fn = {torch.int32: lib.qs_sketch_i32, torch.float64: lib.qs_sketch_f64}.get(keys.dtype)
    if fn is None:
        raise TypeError("sketch takes int32 or float64 keys")
    _check(fn(keys.data_ptr(), keys.numel(), x.data_ptr(), mm.data_ptr(), smp.data_ptr(), _stream_handle(stream)))
    return x, mm, smp


def mlp_param_count() -> int:
    return load().qs_mlp_param_count()


def mlp_forward(params, x, act=None, stream=None):
    """q = model(x) for x (batch x 1024, float32 CUDA); act (batch x 640) is filled if given."""
    import torch

    lib = load()
    batch = x.shape[0]
    q = torch.empty(batch, 255, dtype=torch.float32, device=x.device)
    _check(lib.qs_mlp_forward(params.data_ptr(), x.data_ptr(), batch, q.data_ptr(), _ptr(act), _stream_handle(stream)))
    return q


def mlp_backward(params, x, t, act, work, grad, loss=None, stream=None) -> None:
    lib = load()
    _check(lib.qs_mlp_backward(params.data_ptr(), x.data_ptr(), t.data_ptr(), act.data_ptr(), x.shape[0],
                               work.data_ptr(), grad.data_ptr(), _ptr(loss), _stream_handle(stream)))


def mlp_adam(params, grad, m, v, step: int, lr: float, stream=None) -> None:
    lib = load()
    _check(lib.qs_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), int(step), float(lr),
                           _stream_handle(stream)))


def sort_host(keys, values=None, stream=None) -> None:
    """qs_sort_host_*: sorts host (numpy) arrays in place through the GPU."""
    import numpy as np

    lib = load()
    s = _stream_handle(stream)
    if not keys.flags.c_contiguous:
        raise ValueError("keys must be C-contiguous")
    n = keys.size
    p = ctypes.c_void_p(keys.ctypes.data)
    if values is not None:
        if keys.dtype != np.int32 or values.dtype != np.int32 or values.size != n or not values.flags.c_contiguous:
            raise ValueError("key/value host sort takes contiguous int32 arrays of equal length")
        _check(lib.qs_sort_host_kv(p, ctypes.c_void_p(values.ctypes.data), n, s))
    elif keys.dtype == np.int32:
        _check(lib.qs_sort_host_i32(p, n, s))
    elif keys.dtype == np.float64:
        _check(lib.qs_sort_host_f64(p, n, s))
    else:
        raise TypeError(keys.dtype)


def reserve(n: int, kind: str) -> None:
    _check(load().qs_reserve(int(n), KIND[kind]))


def release() -> None:
    load().qs_release()


def set_option(name: str, value: int) -> None:
    _check(load().qs_set_option(OPTION[name], int(value)))


def get_option(name: str) -> int:
    v = ctypes.c_int64(0)
    _check(load().qs_get_option(OPTION[name], ctypes.byref(v)))
    return v.value


def stats() -> dict:
    st = Stats()
    _check(load().qs_get_stats(ctypes.byref(st)))
    out = {name: getattr(st, name) for name, _ in Stats._fields_}
    out["driver_cycles"] = list(st.driver_cycles)
    return out


def version() -> int:
    return load().qs_version()

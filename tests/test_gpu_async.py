"""The asynchronous sort boundary: qs_sort_* and qs_sort_segmented_* return
once their work is enqueued (Algorithm 3's sort is a plain call with no
result), qs_sync_status() is the synchronisation point, and a device-side
failure is reported exactly once -- by qs_sync_status() or by the next call
that finds the failed call finished.  Calls on different streams are ordered
on the shared workspace.  Outputs are compared with the oracle."""
import ctypes

import numpy as np
import pytest

import synth
from qs_testutil import assert_keys_equal, assert_kv_sorted_equal, oracle_sort, qs_gpu, to_dev

pytestmark = pytest.mark.gpu


def _handle(stream):
    return ctypes.c_void_p(stream.cuda_stream)


def test_c_abi_sorts_return_before_sync_and_sync_status_is_ok():
    """Straight through ctypes: qs_sort_* returns QS_OK after enqueueing,
    qs_sync_status returns QS_OK, and every array is sorted."""
    import torch

    qs = qs_gpu()
    lib = qs.load()
    stream = torch.cuda.Stream()
    xs = [synth.uniform_i32(300_001 + 17 * i, 600 + i) for i in range(6)]
    ds = [to_dev(x) for x in xs]
    fs = synth.uniform_f64(200_003, 610)
    df = to_dev(fs)
    kk, kv = synth.kv_config("uniform", 150_001, 611)
    dk, dv = to_dev(kk), to_dev(kv)
    torch.cuda.synchronize()
    h = _handle(stream)
    for d in ds:
        assert lib.qs_sort_i32(ctypes.c_void_p(d.data_ptr()), d.numel(), h) == 0
    assert lib.qs_sort_f64(ctypes.c_void_p(df.data_ptr()), df.numel(), h) == 0
    assert lib.qs_sort_kv(ctypes.c_void_p(dk.data_ptr()), ctypes.c_void_p(dv.data_ptr()), dk.numel(), h) == 0
    assert lib.qs_sync_status(h) == 0
    for x, d in zip(xs, ds):
        assert_keys_equal(d.cpu().numpy(), oracle_sort(x))
    assert_keys_equal(df.cpu().numpy(), oracle_sort(fs))
    ok, ov = oracle_sort(kk, kv)
    assert_kv_sorted_equal(kk, kv, dk.cpu().numpy(), dv.cpu().numpy(), ok, ov)
    st = qs.stats()  # the last call's device counters, read at qs_sync_status
    assert st["n"] == 150_001 and st["leaf_keys"] + st["copy_keys"] > 0


def test_async_sorts_on_two_streams_are_ordered():
    """Sorts issued without waiting on two streams share one workspace; the
    library orders them on the GPU, so both results are right."""
    import torch

    qs = qs_gpu()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    xs = [synth.uniform_f64(400_001 + i, 620 + i) for i in range(8)]
    ds = [to_dev(x) for x in xs]
    torch.cuda.synchronize()
    for i, d in enumerate(ds):
        qs.sort(d, stream=s1 if i % 2 == 0 else s2, sync=False)
    qs.sync_status(s1)
    qs.sync_status(s2)
    torch.cuda.synchronize()
    for x, d in zip(xs, ds):
        assert_keys_equal(d.cpu().numpy(), oracle_sort(x))


def test_async_segmented_sorts_then_one_sync():
    import torch

    qs = qs_gpu()
    stream = torch.cuda.Stream()
    keys, offs = [], []
    for r in range(3):
        sizes = synth.segment_sizes(150, 630 + r, 16, 1 << 14)
        o = np.zeros(151, dtype=np.int64)
        np.cumsum(sizes, out=o[1:])
        offs.append(o)
        keys.append(synth.uniform_i32(int(o[-1]), 640 + r))
    dk = [to_dev(k) for k in keys]
    do = [to_dev(o) for o in offs]
    torch.cuda.synchronize()
    for k, o in zip(dk, do):
        qs.sort_segmented(k, o, stream=stream, sync=False)
    qs.sync_status(stream)
    for k, o, d in zip(keys, offs, dk):
        got = d.cpu().numpy()
        for i in range(0, 150, 7):
            a, b = int(o[i]), int(o[i + 1])
            assert_keys_equal(got[a:b], oracle_sort(k[a:b]))


def test_async_failure_reported_by_sync_status_once():
    """A capacity overflow of an asynchronous sort: the call itself returns
    QS_OK, qs_sync_status reports QS_ERR_CAPACITY once, and the next sort is
    right."""
    import torch

    qs = qs_gpu()
    stream = torch.cuda.Stream()
    x = synth.uniform_i32(1 << 20, 650)
    qs.set_option("task_cap", 1)
    try:
        d = to_dev(x)
        torch.cuda.synchronize()
        qs.sort(d, stream=stream, sync=False)  # enqueued; no error yet
        with pytest.raises(qs.QSError) as e:
            qs.sync_status(stream)
        assert e.value.code == -6
        qs.sync_status(stream)  # reported once: nothing left to report
    finally:
        qs.set_option("task_cap", 0)
    d = to_dev(x)
    qs.sort(d, stream=stream)
    assert_keys_equal(d.cpu().numpy(), oracle_sort(x))


def test_async_failure_reported_by_the_next_call():
    """A failed asynchronous sort that has finished is reported by the next
    call, which then does nothing (its array is untouched); the call after it
    sorts normally."""
    import torch

    qs = qs_gpu()
    stream = torch.cuda.Stream()
    x = synth.uniform_i32(1 << 20, 660)
    y = synth.uniform_i32(500_001, 661)
    qs.set_option("task_cap", 1)
    try:
        d = to_dev(x)
        torch.cuda.synchronize()
        qs.sort(d, stream=stream, sync=False)
        stream.synchronize()  # the failed call has finished
    finally:
        qs.set_option("task_cap", 0)
    dy = to_dev(y)
    torch.cuda.synchronize()
    with pytest.raises(qs.QSError) as e:
        qs.sort(dy, stream=stream, sync=False)
    assert e.value.code == -6
    assert "earlier asynchronous call" in str(e.value)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dy.cpu().numpy(), y)  # untouched
    qs.sort(dy, stream=stream)
    assert_keys_equal(dy.cpu().numpy(), oracle_sort(y))


def test_async_timeout_reported_and_recovers():
    """With a wait limit of 0 an asynchronous sort's waits run out: the call
    returns QS_OK, qs_sync_status reports QS_ERR_TIMEOUT, and the library
    (look-back words and ticket owners cleaned on the device) sorts the next
    array right without the host having cleared anything in between."""
    import torch

    qs = qs_gpu()
    stream = torch.cuda.Stream()
    x = synth.uniform_f64(1 << 20, 670)
    y = synth.uniform_f64(700_001, 671)
    d, dy = to_dev(x), to_dev(y)
    qs.reserve(1 << 20, "f64")  # no workspace growth (cudaFree synchronises) inside the two calls
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(100_000_000)  # holds the stream, so both sorts are enqueued before either runs
    qs.set_option("wait_limit_ns", 0)
    try:
        qs.sort(d, stream=stream, sync=False)
    finally:
        qs.set_option("wait_limit_ns", 2_000_000_000)
    qs.sort(dy, stream=stream, sync=False)  # issued before anyone looked at the failure
    with pytest.raises(qs.QSError) as e:
        qs.sync_status(stream)
    assert e.value.code == -5
    assert "earlier asynchronous call" in str(e.value)
    assert_keys_equal(dy.cpu().numpy(), oracle_sort(y))
    d = to_dev(x)
    qs.sort(d, stream=stream)
    assert_keys_equal(d.cpu().numpy(), oracle_sort(x))


def test_sync_option_makes_sorts_synchronous():
    import torch

    qs = qs_gpu()
    x = synth.uniform_i32(1 << 20, 680)
    qs.set_option("task_cap", 1)
    qs.set_option("sync", 1)
    try:
        d = to_dev(x)
        torch.cuda.synchronize()
        with pytest.raises(qs.QSError) as e:
            qs.sort(d, sync=False)  # the C call itself returns the error
        assert e.value.code == -6
    finally:
        qs.set_option("task_cap", 0)
        qs.set_option("sync", 0)
    qs.sync_status()

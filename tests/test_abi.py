"""CPU-only checks of the C-ABI library: it builds, loads, exports every entry
point that include/qs.h declares, and its host-side argument checks return the
documented status codes.  No call here reaches a kernel."""
import ctypes

import pytest

import paper_1704_08579_gb300 as qs
from paper_1704_08579_gb300 import build as qs_build


@pytest.fixture(scope="module")
def lib():
    qs_build.build()
    return qs.load()


def test_exports_every_declared_function(lib):
    names = qs.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_options(lib):
    assert lib.qs_version() >= 100
    assert lib.qs_set_option(999, 1) == -1
    assert lib.qs_set_option(qs.OPTION["wait_limit_ns"], -5) == -1
    assert lib.qs_set_option(qs.OPTION["profile"], 0) == 0


def test_host_argument_checks(lib):
    null = ctypes.c_void_p(0)
    assert lib.qs_sort_i32(null, 0, null) == 0          # n == 0 is a no-op
    assert lib.qs_sort_f64(null, 1, null) == 0          # n == 1 is a no-op
    assert lib.qs_partition_i32(null, 0, 5, null) == 0  # empty split
    assert lib.qs_sort_i32(null, -1, null) == -1
    assert b"out of range" in lib.qs_last_error()
    assert lib.qs_sort_kv(null, null, -3, null) == -1
    assert lib.qs_partition_f64(null, (1 << 38) + 1, 0.0, null) == -1
    assert lib.qs_sort_i32(null, 10, null) == -1        # null pointer with n > 0
    assert b"null" in lib.qs_last_error()
    assert lib.qs_sort_f64(ctypes.c_void_p(4), 10, null) == -2  # misaligned double pointer
    assert lib.qs_reserve(10, 7) == -1
    st = qs.stats()
    assert set(st) >= {"part_tasks", "part_keys", "leaf_keys", "ms_driver"}


def test_binding_rejects_bad_dtypes():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        qs.sort(torch.zeros(4, dtype=torch.float32))

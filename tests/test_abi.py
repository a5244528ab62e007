"""CPU-only checks of the C-ABI library: it builds, loads, exports every entry
point that include/qs.h declares, and its host-side argument checks return the
documented status codes.  No call here reaches a kernel."""
import ctypes
import os
import re

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


def test_option_value_ranges(lib):
    """Every option's documented range (include/qs.h); an out-of-range value
    returns QS_ERR_INVALID_ARG and leaves the option alone."""
    opt = qs.OPTION
    for v in (0, 1, 2):
        assert lib.qs_set_option(opt["profile"], v) == 0
    for v in (-1, 3):
        assert lib.qs_set_option(opt["profile"], v) == -1
    for v in (0, 1):
        assert lib.qs_set_option(opt["ordered"], v) == 0
    for v in (-1, 2):
        assert lib.qs_set_option(opt["ordered"], v) == -1
    for v in (0, 8, 16, 32):
        assert lib.qs_set_option(opt["driver_items"], v) == 0
    for v in (-1, 65):
        assert lib.qs_set_option(opt["driver_items"], v) == -1
    for name in ("leaf_max", "small_max"):
        for v in (0, 32, 512, 4096):
            assert lib.qs_set_option(opt[name], v) == 0
        for v in (-1, 16, 48, 1000):
            assert lib.qs_set_option(opt[name], v) == -1
    assert lib.qs_set_option(opt["driver_ctas"], -1) == -1
    assert lib.qs_set_option(opt["driver_ctas"], (1 << 20) + 1) == -1
    assert lib.qs_set_option(opt["task_cap"], -1) == -1
    for v in (0, 1):
        assert lib.qs_set_option(opt["sync"], v) == 0
    for v in (-1, 2):
        assert lib.qs_set_option(opt["sync"], v) == -1
    for name in ("profile", "ordered", "driver_items", "leaf_max", "small_max", "driver_ctas", "task_cap", "sync"):
        assert lib.qs_set_option(opt[name], 0) == 0
    assert lib.qs_set_option(opt["wait_limit_ns"], 2_000_000_000) == 0


def test_get_option_reads_back_what_was_set(lib):
    for name, v in (("leaf_max", 1024), ("small_max", 64), ("driver_items", 8), ("sync", 1), ("ordered", 1)):
        assert lib.qs_set_option(qs.OPTION[name], v) == 0
        assert qs.get_option(name) == v
        assert lib.qs_set_option(qs.OPTION[name], 0) == 0
        assert qs.get_option(name) == 0
    assert qs.get_option("wait_limit_ns") == 2_000_000_000
    assert lib.qs_get_option(999, ctypes.byref(ctypes.c_int64())) == -1
    assert lib.qs_get_option(qs.OPTION["sync"], None) == -1


def test_option_names_match_header():
    """The binding's option numbers are the header's QS_OPT_* values."""
    import re

    text = open(qs.HEADER).read()
    found = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"QS_OPT_([A-Z_]+)\s*=\s*(\d+)", text)}
    assert found == qs.OPTION


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
    assert lib.qs_partition_f64(null, 10, float("nan"), null) == -1  # no side is defined for a NaN pivot
    assert b"NaN" in lib.qs_last_error()
    assert lib.qs_reserve(10, 7) == -1
    # The no-allocation partition checks its arguments before any CUDA call.
    cap = 1 << int(re.search(r"#define QS_NOALLOC_MAX_N \(1 << (\d+)\)", open(qs.HEADER).read()).group(1))
    assert lib.qs_partition_i32_noalloc(null, 0, 5, null) == 0
    assert lib.qs_partition_i32_noalloc(null, cap + 1, 5, null) == -1
    assert lib.qs_partition_i32_noalloc(null, -1, 5, null) == -1
    assert lib.qs_partition_i32_noalloc(null, 10, 5, null) == -1
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(6), 10, 5, null) == -2
    st = qs.stats()
    assert set(st) >= {"part_tasks", "part_keys", "leaf_keys", "ms_driver"}


def test_binding_rejects_bad_dtypes():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        qs.sort(torch.zeros(4, dtype=torch.float32))


def test_stats_layout_matches_header(tmp_path):
    """The binding's qs_stats mirror has the header's size and field offsets
    (qs_get_stats writes sizeof(qs_stats) bytes into the caller's struct)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [name for name, _ in qs.Stats._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"qs.h\"\nint main(void) {\n"
                   "  printf(\"size %zu\\n\", sizeof(qs_stats));\n"
                   + "".join("  printf(\"%s %%zu\\n\", offsetof(qs_stats, %s));\n" % (f, f) for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(qs.HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(qs.Stats)
    for f in fields:
        assert int(out[f]) == getattr(qs.Stats, f).offset, f


def test_no_cpu_fallback(monkeypatch):
    """CPU tensors are refused (nothing sorts them on the host), and without
    the built library every call raises instead of running anything else."""
    torch = pytest.importorskip("torch")
    x = torch.arange(10, 0, -1, dtype=torch.int32)
    before = x.clone()
    with pytest.raises(ValueError):
        qs.sort(x)
    with pytest.raises(ValueError):
        qs.partition(x, 5)
    assert torch.equal(x, before)
    monkeypatch.setattr(qs, "_lib", None)
    monkeypatch.setattr(qs, "LIB_PATH", os.path.join(os.path.dirname(qs.LIB_PATH), "missing", "libqs.so"))
    with pytest.raises(RuntimeError, match="not built"):
        qs.load()
    with pytest.raises(RuntimeError, match="not built"):
        qs.sort(x)


def test_plain_c_caller(tmp_path, lib):
    """The boundary is usable from C alone: a program compiled with gcc against
    include/qs.h and linked with libqs.so calls the entry points that return
    before any CUDA call (version, options, argument checks, last error)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "qs.h"
int main(void) {
    int64_t v = -1;
    if (qs_version() < 100) return 1;
    if (qs_set_option(QS_OPT_SYNC, 1) != QS_OK) return 2;
    if (qs_get_option(QS_OPT_SYNC, &v) != QS_OK || v != 1) return 3;
    if (qs_set_option(QS_OPT_SYNC, 0) != QS_OK) return 4;
    if (qs_sort_i32(NULL, -1, NULL) != QS_ERR_INVALID_ARG) return 5;
    if (strstr(qs_last_error(), "out of range") == NULL) return 6;
    if (qs_sort_f64((double *)8, 0, NULL) != QS_OK) return 7;
    if (qs_partition_kv(NULL, NULL, 0, 0, NULL) != 0) return 8;
    if (qs_sort_f64((double *)4, 10, NULL) != QS_ERR_ALIGN) return 9;
    if (qs_partition_i32_noalloc(NULL, QS_NOALLOC_MAX_N + 1, 0, NULL) != QS_ERR_INVALID_ARG) return 10;
    printf("ok\n");
    return 0;
}
""")
    exe = tmp_path / "caller"
    libdir = os.path.dirname(qs.LIB_PATH)
    subprocess.run([cc, "-I", os.path.dirname(qs.HEADER), str(src), "-o", str(exe), "-L", libdir, "-lqs",
                    "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_header_is_clean_c_and_cxx(tmp_path, lang, std):
    """include/qs.h compiles on its own as strict C99 and C++11, warnings as errors."""
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no compiler")
    src = tmp_path / "hdr.c"
    src.write_text('#include "qs.h"\nint main(void) { return QS_OK; }\n')
    subprocess.run([cc, std, "-x", lang, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(qs.HEADER),
                    str(src), "-o", str(tmp_path / "hdr")], check=True)

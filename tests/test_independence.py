"""Structural checks (CPU): the CUDA path and the oracle share nothing.

The oracle is test infrastructure.  The library (``paper_1704_08579_gb300/``
and ``include/``) must neither import, load nor include anything under
``oracle/``, and the oracle must not include the library's headers or
sources; the seeded input generators (``synth/``) hold no sorting or
partition arithmetic and import neither side.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    out = []
    for dirpath, dirnames, filenames in os.walk(os.path.join(ROOT, sub)):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__", "_lib", "tuning"))]
        out += [os.path.join(dirpath, f) for f in filenames if f.endswith(exts)]
    return out


def _text(path):
    with open(path, encoding="utf-8") as f:
        return f.read()


def test_library_never_reaches_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|qs_oracle|oracle_[a-z0-9_]+\(|liboracle", re.M)
    files = _files("paper_1704_08579_gb300", (".py", ".cu", ".cuh", ".h", ".cpp")) + _files("include", (".h",))
    assert files
    for p in files:
        assert not pat.search(_text(p)), p


def test_oracle_includes_nothing_of_the_library():
    files = _files("oracle", (".py", ".cpp", ".h", ".c"))
    assert files
    for p in files:
        t = _text(p)
        assert not re.search(r"^\s*(import|from)\s+paper_1704_08579_gb300\b", t, re.M), p
        assert "csrc" not in t and "libqs" not in t, p
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', t):
            assert not inc.startswith("qs") and "/" not in inc, (p, inc)


def test_generators_import_neither_side():
    for p in _files("synth", (".py",)):
        t = _text(p)
        assert not re.search(r"^\s*(import|from)\s+(oracle|paper_1704_08579_gb300)\b", t, re.M), p

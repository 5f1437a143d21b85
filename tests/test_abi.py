"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/graph_reduce.h declares.  No GPU needed
(no call here reaches a CUDA compute path)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "graph_reduce.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(graph_reduce_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_08942_gb300 import build as B
    B.build()
    from paper_1812_08942_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("graph_reduce_create", "graph_reduce_smooth", "graph_reduce_affinity",
                     "graph_reduce_aggregate", "graph_reduce_coarsen", "graph_reduce_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_08942_gb300 import binding
    names = _declared()
    out = subprocess.run(["nm", "-D", "--defined-only", binding.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (graph_reduce_\w+)", out))
    for name in names:
        assert name in exported, name
        assert hasattr(lib, name)
    # the Python binding wraps exactly the declared set
    assert sorted(binding.EXPORTED) == names


def test_argument_errors_need_no_gpu(lib):
    from paper_1812_08942_gb300 import binding
    h = ctypes.c_void_p()
    st = lib.graph_reduce_create(ctypes.byref(h), 0, 0, None, None, None, 1, None)
    assert st == binding.GR_EINVAL
    assert b"n must be" in lib.graph_reduce_last_error(None)
    st = lib.graph_reduce_smooth(None, 16, 5, 0.7, 0, 0, 1, None)
    assert st == binding.GR_EINVAL
    lib.graph_reduce_destroy(None)  # NULL-safe


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1812_08942_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "_LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        binding.load()

"""The C-ABI library builds, loads without a GPU, and exports every symbol include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(bridges_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["bridges_find", "bridges_find_ctx", "bridges_find_host", "bridges_ctx_create",
                 "bridges_ctx_destroy", "bridges_certificate", "bridges_from_forest"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2108_07346_gb300 import build

    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2108_07346_gb300 as pb

    assert set(declared_functions()) <= set(pb.exported_symbols())


def test_status_strings_without_gpu():
    import paper_2108_07346_gb300 as pb

    assert pb.status_string(-2).startswith("vertex id")
    assert pb.status_string(0) == "ok"


def test_ctx_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2108_07346_gb300 as pb

    lib = pb.load()
    assert not lib.bridges_ctx_create(0, 0, None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the compiled library the binding raises instead of computing
    anything on the CPU."""
    import paper_2108_07346_gb300 as pb
    from paper_2108_07346_gb300 import build

    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(pb, "_lib", None)
    with pytest.raises(RuntimeError, match="libbridges.so not found"):
        pb.load(build_if_missing=False)

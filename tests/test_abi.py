"""The C-ABI library builds, loads without a GPU, and exports every symbol include/*.h declares."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

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


# Entry points that report "nothing" as 0 rather than as an error status.
_ZERO_WHEN_EMPTY = {"bridges_ctx_ap_stage_ms", "bridges_ctx_ap_stage_ms_history", "bridges_ctx_last_config",
                    "bridges_ctx_launches", "bridges_ctx_stage_ms", "bridges_ctx_stage_ms_history",
                    "bridges_server_stats", "bridges_workspace_bytes", "bridges_articulation_workspace_bytes"}
# Creation calls, the status table, and the two calls without a handle, for which all-zero
# arguments form a valid request rather than an error.
_NOT_HANDLE_CALLS = {"bridges_ctx_create", "bridges_ctx_create_ws", "bridges_server_create", "bridges_inc_create",
                     "bridges_status_string", "bridges_find", "bridges_find_noalloc"}


def test_null_handles_are_rejected_without_touching_a_gpu():
    """Every call on a context, server or incremental handle checks the handle before anything
    else: a null handle (all other arguments zero) gives BRIDGES_EINVAL, or 0 where the call
    reports a count or a size, and the destroy calls do nothing."""
    import paper_2108_07346_gb300 as pb

    lib = pb.load()
    checked = 0
    for name, (restype, argtypes) in sorted(pb._SIGS.items()):
        if name in _NOT_HANDLE_CALLS:
            continue
        args = [None if t is ctypes.c_void_p or hasattr(t, "contents") else 0 for t in argtypes]
        got = getattr(lib, name)(*args)
        if restype is None:
            assert got is None, name
        elif name in _ZERO_WHEN_EMPTY:
            assert got == 0, name
        else:
            assert got == -1, (name, got)
        checked += 1
    assert checked >= 30


@pytest.mark.skipif(not shutil.which("gcc"), reason="needs gcc")
def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and field offsets, as a C
    compiler lays them out (a field added, dropped or retyped on one side only would shift the
    rest)."""
    import paper_2108_07346_gb300 as pb

    pairs = [("bridges_opts", pb.Opts), ("bridges_batch_plan", pb.BatchPlan), ("bridges_request", pb.Request)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "bridges.h")}"',
             "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for cname, cls in pairs:
        assert int(got[f"{cname} size"]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname} {fname}"]) == getattr(cls, fname).offset, (cname, fname)

"""Planted mistakes in the oracle, on the CPU: the pins must reject each one.

Each mutant is the oracle's C source with one plausible error (a dropped term, a wrong
comparison, a skipped step), built with the same gcc command into a temporary library and
swapped in for the real one.  The pins of test_oracle (hand-derived fixtures, closed forms,
brute force by definition, certificate invariants) then run against it, and at least one must
fail.  The unmodified source, built the same way, must pass them all, so a broken harness
cannot make every mutant look caught.

The mutants cover Alg. 1 (bridge DFS), Alg. 2 (the two forests), the Sec. 3 pipeline
(partition and merge), the independent checks (Schmidt chains, two-edge components) and the
articulation-point routine.  None of them can write outside its buffers: each only changes
which edges or vertices are counted.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle as T
from conftest import golden_names

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# name: (text in oracle.c, replacement, which occurrence (0-based), passage it breaks)
MUTANTS = {
    "parent skipped by vertex": (
        "if (e == st_pe[sp]) continue; /* the edge we came in by */",
        "if (sp > 0 && w == st_v[sp - 1]) continue;", 0, "Alg. 1"),
    ">= in the bridge test": (
        "if (low[x] > disc[p]) keys[nb++] = pair_key(p, x);",
        "if (low[x] >= disc[p]) keys[nb++] = pair_key(p, x);", 0, "Alg. 1"),
    "child low not folded into parent": (
        "if (low[x] < low[p]) low[p] = low[x];", ";", 0, "Alg. 1"),
    "DFS from vertex 0 only": (
        "  for (int32_t s = 0; s < V; s++) {\n    if (disc[s]) continue;",
        "  for (int32_t s = 0; s < (V > 0 ? 1 : 0); s++) {\n    if (disc[s]) continue;", 0, "Alg. 1"),
    "F' drawn from all edges": (
        "    if (in_f[i]) continue;\n", "", 0, "Alg. 2"),
    "merge partner dropped": (
        "      if (i + s < M) {\n", "      if (0) {\n", 0, "Sec. 3 merge phases"),
    "last edge of each chunk lost": (
        "int64_t lo = (E * (int64_t)i) / M, hi = (E * (int64_t)(i + 1)) / M;",
        "int64_t lo = (E * (int64_t)i) / M, hi = (E * (int64_t)(i + 1)) / M;\n    if (hi > lo) hi--;", 0,
        "Sec. 3 partition"),
    "chain walk stops after one step": (
        "      while (!visited[w]) {", "      if (!visited[w]) {", 0, "Schmidt chains"),
    "bridges kept in two-edge components": (
        "    if (bsearch(&k, keys, (size_t)nb, sizeof(uint64_t), cmp_u64)) continue;\n", "", 0,
        "two-edge components"),
    "root with one child a cut vertex": (
        "if (nchild[s] >= 2) ap[s] = 1;", "if (nchild[s] >= 1) ap[s] = 1;", 0, "articulation points"),
    "> in the cut-vertex test": (
        "if (sp - 1 > 0 && low[x] >= disc[p]) ap[p] = 1;", "if (sp - 1 > 0 && low[x] > disc[p]) ap[p] = 1;", 0,
        "articulation points"),
    "child low not folded (cut vertices)": (
        "if (low[x] < low[p]) low[p] = low[x];", ";", 1, "articulation points"),
}


def pins():
    """The pins of test_oracle that take no fixture, parameter loops spelled out."""
    methods = sorted(T.ALL_METHODS)
    return [
        ("golden fixtures", lambda: [T.test_golden(n, m) for n in golden_names() for m in methods]),
        ("golden cut vertices", lambda: [T.test_golden_cut_vertices(n) for n in golden_names()]),
        ("closed forms", lambda: [T.test_closed_forms(m) for m in methods]),
        ("random multigraphs, three methods", T.test_random_multigraphs_agree),
        ("sparse trees plus edges", T.test_sparse_random_trees_plus_edges),
        ("planted counts", T.test_planted_counts_small),
        ("certificate invariants", T.test_certificate_invariants_random),
        ("certificate cut property", T.test_certificate_cut_property),
        ("streaming certificate", T.test_streaming_certificate_equals_two_pass),
        ("two-edge components, brute force", T.test_two_edge_components_brute),
        ("two-edge components, closed forms", T.test_two_edge_components_closed_forms),
        ("cut vertices, brute force and closed forms", T.test_articulation_points_brute_and_closed_forms),
        ("block certificate", T.test_block_certificate_articulation_points),
    ]


def replace_nth(text, old, new, n):
    at = -1
    for _ in range(n + 1):
        at = text.index(old, at + 1)
    return text[:at] + new + text[at + len(old):]


def build_variant(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    lib = tmp_path / f"lib{name}.so"
    src.write_text(text)
    cmd = oracle._build.command()
    cmd[cmd.index(oracle._build.SRC)] = str(src)
    cmd[cmd.index(oracle._build.LIB)] = str(lib)
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(lib)


def failing_pins(monkeypatch, lib):
    """Names of the pins that fail with the oracle library at `lib` swapped in."""
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: lib)
    failed = []
    for name, check in pins():
        try:
            check()
        except AssertionError:
            failed.append(name)
    return failed


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


def test_unmodified_source_passes_every_pin(monkeypatch, tmp_path, source):
    lib = build_variant(tmp_path, "control", source)
    assert failing_pins(monkeypatch, lib) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, tmp_path, source, mutant):
    old, new, nth, passage = MUTANTS[mutant]
    assert source.count(old) > nth, f"the text to mutate ({passage}) is no longer in oracle.c"
    text = replace_nth(source, old, new, nth)
    lib = build_variant(tmp_path, "mutant", text)
    assert failing_pins(monkeypatch, lib), f"no pin rejects the mutant '{mutant}' ({passage})"

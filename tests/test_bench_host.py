"""Host-side helpers of bench.py that need no GPU: the source hash that decides whether a
stored DRAM-traffic figure still describes the kernel's code, the served bench's request stream and the
reference arm's JSON line."""
import os

import pytest

import bench


def test_code_only_strips_comments_and_keeps_literals():
    src = ("int a = 1; // note\n/* block\n comment */ int b = 2;\n\n"
           "  const char* s = \"// not a comment\";\nchar c = '/';\n")
    assert bench.code_only(src).splitlines() == [
        "int a = 1;", " int b = 2;", "  const char* s = \"// not a comment\";", "char c = '/';"]


def test_comment_edits_keep_the_hash_and_code_edits_change_it(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2108_07346_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("int f() { return 1; } // one\n")
    h0 = bench.sources_sha(("k.cu",))
    (csrc / "k.cu").write_text("// a new comment\nint f() { return 1; }   /* another */\n\n")
    assert bench.sources_sha(("k.cu",)) == h0
    (csrc / "k.cu").write_text("int f() { return 2; }\n")
    assert bench.sources_sha(("k.cu",)) != h0


def test_stored_traffic_figures_name_their_sources():
    """Each stored figure carries the hash of the sources it was captured on; bench.py reports it
    only while the current sources hash the same."""
    for table, key in ((bench.TRAFFIC, "certify_sha"), (bench.AP_TRAFFIC, "blocks_sha"),
                       (bench.FUSED_TRAFFIC, "blocks_sha")):
        assert len(table[key]) == 16 and table["bytes_per_edge"] > 8.0


def test_request_stream_hands_out_requests_in_order(monkeypatch):
    """The served bench's producer threads generate out of order; the consumer gets request
    first, first + 1, ... and the byte budget is returned on release."""
    import random
    import time as _time
    from types import SimpleNamespace

    import graphgen

    def fake(specs, dev, stream=None):
        _time.sleep(random.random() * 0.002)
        return [SimpleNamespace(E=int(spec.core_vertices), seed=spec.seed) for spec in specs]

    monkeypatch.setattr(graphgen, "generate_device_many", fake)
    rs = bench.RequestStream("cpu", 10, 200, ahead=16, max_bytes=1 << 40, threads=3, batch=5)
    got = []
    for _ in range(200):
        i, g = rs.get()
        assert g.seed == graphgen.workload_spec("served", 4, i).seed
        got.append(i)
        rs.release(g)
    assert got == list(range(10, 210)) and rs.bytes == 0 and rs.error is None


def test_request_stream_reports_a_failed_generation(monkeypatch):
    import graphgen

    def boom(specs, dev, stream=None):
        raise ValueError("no device")

    monkeypatch.setattr(graphgen, "generate_device_many", boom)
    rs = bench.RequestStream("cpu", 0, 8, threads=2)
    with pytest.raises(RuntimeError, match="request generation failed"):
        rs.get()


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` runs the oracle on the host cores (no GPU needed) and prints one
    JSON line with the keys both arms share, its own CPU baseline and a zero-copy e2e figure."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "2",
                        "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=300, check=True)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GE/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "small" and d["config"]["sample_edges_per_step"] == d["config"]["E"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

"""Host-side helpers of bench.py that need no GPU: the source hash that decides whether a
stored DRAM-traffic figure still describes the kernel's code."""
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

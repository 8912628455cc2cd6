"""Host logic of the benchmark (no GPU): the kernel-source digest that keys
recorded ncu counters ignores comments and whitespace but not code, and the
z-pass roofline is reported against the issue roof only while the record's
digest matches the sources."""
import bench


def test_code_text_strips_comments_only():
    a = "int x = 1; // one\n/* block\n comment */ float y = 2.0f;\n"
    b = "int x = 1;\n\n   float y = 2.0f;   // another note\n"
    assert bench.code_text(a) == bench.code_text(b) == "int x = 1; float y = 2.0f;"
    assert bench.code_text("int x = 2;") != bench.code_text("int x = 1;")


def test_digest_follows_code_not_comments():
    base = {f: "int f_%d(){return %d;}\n" % (i, i) for i, f in enumerate(bench.TRAFFIC_SOURCES)}
    d0 = bench.sources_digest(lambda f: base[f])
    commented = {f: "// header\n" + t + "/* trailing */\n" for f, t in base.items()}
    assert bench.sources_digest(lambda f: commented[f]) == d0
    changed = dict(base)
    changed[bench.TRAFFIC_SOURCES[0]] = "int f_0(){return 7;}\n"
    assert bench.sources_digest(lambda f: changed[f]) != d0


def test_roofline_uses_the_record_only_for_matching_sources(monkeypatch):
    passes = {"z": {"ms_per_launch": 6.8}}
    rec = {"sources": bench.sources_digest(), "bytes_per_launch": 16.7e9, "warp_inst_per_launch": 6.9e9}
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("k_pass_z", 768, False), rec)
    r = bench.roofline("z", 6.8, 768, False, True, 2400.0, 6669.0, "measured",
                       {"sm_max_mhz": 2070.0}, passes)
    assert r["bound"] == "alu" and abs(r["frac"] - 6.9e9 / 6.8e-3 / (152 * 4 * 2.07e9)) < 1e-9
    assert r["traffic"] == 16.7e9
    stale = dict(rec, sources="0000000000000000")
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("k_pass_z", 768, False), stale)
    r = bench.roofline("z", 6.8, 768, False, True, 2400.0, 6669.0, "measured",
                       {"sm_max_mhz": 2070.0}, passes)
    assert r["bound"] == "hbm" and r["traffic"] is None

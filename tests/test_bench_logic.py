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
    n3 = 768 ** 3
    rec = {"sources": bench.sources_digest(), "bytes_per_particle": 16.7e9 / n3,
           "warp_inst_per_particle": 6.9e9 / n3, "measured_at": "test"}
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("k_pass_z", 768, False), rec)
    r = bench.roofline("z", 6.8, 768, False, True, 2400.0, 6669.0, "measured",
                       {"sm_max_mhz": 2070.0}, passes)
    assert r["bound"] == "alu" and abs(r["frac"] - 6.9e9 / 6.8e-3 / (152 * 4 * 2.07e9)) < 1e-9
    assert abs(r["traffic"] - 16.7e9) < 1.0
    stale = dict(rec, sources="0000000000000000")
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("k_pass_z", 768, False), stale)
    r = bench.roofline("z", 6.8, 768, False, True, 2400.0, 6669.0, "measured",
                       {"sm_max_mhz": 2070.0}, passes)
    assert r["bound"] == "hbm" and r["traffic"] is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` runs the oracle on the host cores (no GPU)
    and prints one JSON line with the keys the benchmark contract names."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT

"""bench.py reports the DRAM traffic of a kernel from profiles/traffic.json
only while the sources listed with the capture still hash to the recorded
value: a capture of an older kernel version reads as null."""

import importlib.util
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path):
    """A copy of the recorded sources and the record under tmp_path."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for kernel in rec.values():
        if not isinstance(kernel, dict):
            continue
        for entry in kernel.values():
            for src in entry.get("sources", []):
                dst = tmp_path / src
                dst.parent.mkdir(parents=True, exist_ok=True)
                shutil.copyfile(os.path.join(ROOT, src), dst)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return rec


def test_recorded_traffic_matches_current_sources(tmp_path, monkeypatch):
    b = _bench()
    rec = _tree(tmp_path)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    entry = rec["large_projection_fp64"]["ball_pop_n20"]
    got = b.recorded_traffic("large_projection_fp64", "ball_pop_n20")
    assert got == entry["dram_bytes_per_launch"] > 0
    # the per-kernel figures add up to the projection's
    assert sum(entry["per_kernel"].values()) == entry["dram_bytes_per_launch"]
    assert b.recorded_traffic("large_projection_fp64", "no_such_workload") is None
    assert b.recorded_traffic("no_such_kernel", "ball_pop_n20") is None


def test_recorded_traffic_withheld_after_a_source_change(tmp_path, monkeypatch):
    b = _bench()
    rec = _tree(tmp_path)
    src = rec["large_projection_fp64"]["ball_pop_n20"]["sources"][0]
    with open(tmp_path / src, "a") as f:
        f.write("\n// edited after the capture\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.recorded_traffic("large_projection_fp64", "ball_pop_n20") is None

"""The JSON line of bench.py (CPU): every key the benchmark contract asks for,
with the types it asks for, from the line-assembly function with synthetic
numbers; the reference arm's line from a short oracle run."""
import argparse
import contextlib
import io
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TOP = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
       "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
       "config": dict, "roofline": dict, "e2e": dict, "gpu_launches": int, "clocks": dict,
       "cpu_baseline": dict}


def _line(fn):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        fn()
    return json.loads(buf.getvalue().strip().splitlines()[-1])


def test_grid_line_has_the_contract_keys(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = argparse.Namespace(steps=10, warmup=3)
    e2e = {"value": 1.0e11, "unit": "updates/s", "h2d_bytes_per_step": 524.0, "d2h_bytes_per_step": 4194304}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}
    cpu = {"value": 2.0e7, "unit": "updates/s", "cores": 16, "kind": "oracle", "sample": "window"}
    d = _line(lambda: bench.finish(args, 0, 1, 0.004, 1.2e11, 2700.0, 6769.4, "measured", 4, 768, 40,
                                   e2e, clocks, cpu, bench.Ranks("gloo"), {"stream_collide_ms_per_launch": 0.19}))
    for k, t in TOP.items():
        assert k in d and isinstance(d[k], t), k
    assert "vs_baseline" in d and d["vs_baseline"] is None
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "traffic" in r  # measured DRAM bytes while the kernel matches the capture, else null
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["ms_per_step"] == pytest.approx(0.4)


def test_traffic_fingerprint(tmp_path, monkeypatch):
    # measured DRAM traffic is reported only for the grid it was taken on and only
    # while the kernel code is the captured one; comments do not count as code
    assert bench.stage_traffic(160) is None
    assert bench.stage_traffic(256) in (None, bench.STAGE_TRAFFIC["bytes_per_launch"])
    csrc = tmp_path / "paper_1108_5561_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(ROOT, "paper_1108_5561_gb300", "csrc")
    for f in bench.STAGE_TRAFFIC["sources"]:
        (csrc / f).write_text(open(os.path.join(src, f)).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.code_digest(bench.STAGE_TRAFFIC["sources"])
    f0 = csrc / bench.STAGE_TRAFFIC["sources"][0]
    f0.write_text("// a new comment\n/* and a block\n comment */\n" + f0.read_text())
    assert bench.code_digest(bench.STAGE_TRAFFIC["sources"]) == d0
    f0.write_text(f0.read_text() + "\nstatic int extra_code = 1;\n")
    assert bench.code_digest(bench.STAGE_TRAFFIC["sources"]) != d0


def test_reference_arm_line(oracle_mod, monkeypatch):
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    d = _line(lambda: bench.reference_arm(args, 0, 1))
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["metric"] == "site-population updates/s"


def test_run_record_appends_jsonl(tmp_path, monkeypatch):
    path = tmp_path / "runs.jsonl"
    monkeypatch.setattr(bench, "RECORD", str(path))
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    for _ in range(2):
        d = _line(lambda: bench.reference_arm(args, 0, 1))
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(rows) == 2 and rows[-1] == d

"""The benchmark's JSON line, checked on the CPU through its reference arm.

`bench.py --impl reference` times the oracle on the host cores, so it runs
without a GPU; its line must carry the keys a reader of the benchmark relies
on, with the reference arm's own cpu_baseline and e2e objects."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("scale_f64_n8")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pipe_ceiling_takes_the_slowest_pipe(tmp_path, monkeypatch):
    # per-argument work on each pipe / its measured rate; the largest time bounds the kernel
    bench = _bench_module()
    rec = {"per_arg": {"fp64_dfma": 1.0, "alu": 10.0, "fmaheavy_imad": 4.0, "inst": 20.0},
           "sources": ["bench.py"], "sha256": bench._sources_sha(["bench.py"])}
    monkeypatch.setattr(bench, "_pipes", lambda: {"k": rec, "stale": dict(rec, sha256="0" * 64)})
    rates = {"fma": 32e9 * 16, "alu_warp": 600e9, "imad_warp": 300e9, "sms": 152}
    count, secs = 1 << 20, 2e-4
    c = bench.pipe_ceiling("k", count, secs, rates, 2.07e9)
    t = {"fp64": count / 16e9, "alu": 10 * count / 600e9, "fmaheavy": 4 * count / 300e9,
         "issue": 20 * count / (4 * 152 * 2.07e9)}
    pipe = max(t, key=t.get)
    assert c["bound_pipe"] == pipe
    assert abs(c["frac"] - t[pipe] / secs) < 1e-3
    assert bench.pipe_ceiling("stale", count, secs, rates, 2.07e9) is None  # sources changed since the capture
    roof = {"achieved": 1.0, "peak": 2.0, "unit": "x", "frac": 0.5, "note": "model"}
    bench.apply_ceiling(roof, c)
    assert roof["frac"] == c["frac"] and roof["fp64_model"]["frac"] == 0.5
    assert abs(roof["achieved"] / roof["peak"] - c["frac"]) < 1e-2


def test_row_errors_measure_every_m():
    import numpy as np

    bench = _bench_module()
    ref = np.array([[1.0, 0.5], [2.0, 1e-310]])
    got = ref * np.array([[1 + 1e-15, 1 - 3e-15], [1, 1]])
    acc = bench.row_errors(got, ref, "f64", 2)
    assert acc["pass"] and abs(acc["max_rel_err_per_m"][1] - 3e-15) < 1e-16
    bad = got.copy()
    bad[0, 0] = 1.0 + 1e-13
    assert not bench.row_errors(bad, ref, "f64", 2)["pass"]
    nan = got.copy()
    nan[1, 0] = np.nan
    assert not bench.row_errors(nan, ref, "f64", 2)["pass"]

"""The benchmark's reference arm on CPU: `bench.py --impl reference` times the
CPU oracle on a bounded sample of the workload and prints one JSON line in
the benchmark's shape (no GPU is used on this arm)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
           "--steps", "2", "--warmup", "3", "--cpu-windows", "200000"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout[-3000:]
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "k-mers/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == 1
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["k"] == 31 and d["config"]["workload"].startswith("tiny")


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_counter_key_ignores_comments_but_not_code(tmp_path):
    """The per-key ncu counters are keyed to the kernel source's code: a comment
    or whitespace edit keeps the key, any code edit changes it."""
    b = _bench_module()
    src = "// header\nint f(int x) {  /* doubled */\n    return 2 * x;  // twice\n}\n"
    a = tmp_path / "a.cu"
    a.write_text(src)
    base = b.source_sha(str(a))
    a.write_text("// another header\n\nint f(int x) {\n    return 2 *   x;  // times two\n}\n")
    assert b.source_sha(str(a)) == base
    a.write_text(src.replace("2 * x", "3 * x"))
    assert b.source_sha(str(a)) != base

"""Host-side parts of bench.py that need no GPU.

* The code hash that decides whether recorded ncu counters still describe
  the library ignores comments and blank lines but changes with any code.
* The reference arm (the CPU oracle) prints one JSON line with the keys the
  benchmark contract asks for; it runs here on a small cube.
"""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_strips_comments_and_keeps_literals():
    src = ('int a = 1;  // note "q"\n'
           '/* several\n   lines */ const char* s = "a // b /* c */";\n'
           '\n'
           "char c = '/'; double d; /* x */ int e;  \n")
    assert bench.code_only(src) == ('int a = 1;\n'
                                    '  const char* s = "a // b /* c */";\n'
                                    "char c = '/'; double d;   int e;")


def test_code_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2404_02433_b300", "csrc"),
                    root / "paper_2404_02433_b300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    base = bench.src_hash()
    f = root / "paper_2404_02433_b300" / "csrc" / "kernels.cu"
    text = f.read_text()
    f.write_text("// an added comment line\n" + text.replace("\n", "  \n", 3) + "\n/* end */\n")
    assert bench.src_hash() == base
    f.write_text(text + "\nstatic int g_unused_probe = 0;\n")
    assert bench.src_hash() != base


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--n", "48", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--warmup", "2"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0 and "warmup" in out.stderr

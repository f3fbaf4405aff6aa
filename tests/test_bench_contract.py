"""bench.py's host-side contract, on the CPU: the reference arm (the oracle)
prints one JSON line with the keys the harness reads; the algorithmic bytes
per crossing follow the absorber and deposit payloads; the committed DRAM
traffic table parses."""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1101_4127_gb300 import inputs, native  # noqa: E402


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "stromgren_32", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "cell crossings/s" and d["value"] > 0
    assert d["unit"] == "crossings/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_bytes_per_crossing_follow_the_payloads():
    h = inputs.stromgren_32().boxes[0]                 # pure H, isothermal
    hhe = inputs.hhe_blackbody_128(n=8).boxes[0]        # H+He, evolving T
    assert bench.bytes_per_crossing(h, native.CRASH_FP64_PLAIN) == 8 + 8
    assert bench.bytes_per_crossing(hhe, native.CRASH_FP64_PLAIN) == 24 + 32
    assert bench.bytes_per_crossing(hhe, native.CRASH_MIXED) == 12 + 32


def test_traffic_table_rows_parse():
    """Rows: the workloads a capture stands for | k_mixed.cu sha256[:12] |
    DRAM bytes per crossing | the capture it came from."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    rows = [l for l in open(path) if l.startswith("| lognormal")]
    assert rows
    for l in rows:
        c = [x.strip() for x in l.strip().strip("|").split("|")]
        assert re.fullmatch(r"[0-9a-f]{12}", c[1]) and 0 < float(c[2]) < 1000 and c[3]
    ksrc = os.path.join(ROOT, "paper_1101_4127_gb300", "csrc", "k_mixed.cu")
    per = bench.traffic_for("lognormal_512_thin", ksrc)
    assert per is None or per > 0

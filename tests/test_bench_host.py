"""Host-side logic of bench.py, without a GPU: the reference arm's JSON line
(the CPU oracle timed on a sample of the workload) and the source
fingerprint that decides whether a recorded DRAM-traffic figure still
describes the kernel as it is."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line with the keys the
    benchmark contract asks of the reference arm."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-docs", "40"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in r, k
    assert r["metric"] == bench.METRIC and r["unit"] == "docs/s"
    assert r["value"] > 0 and r["higher_is_better"] is True and r["vs_baseline"] is None
    assert r["steps"] == 1 and r["warmup"] == 1 and r["n_gpus"] == 1
    assert r["config"]["workload"].startswith("pes2o_1m")
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert "40 docs" in cb["sample"]
    e2e = r["e2e"]
    assert e2e["value"] == r["value"] and e2e["unit"] == r["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # ms per step and value agree: value counts the sample's documents
    assert abs(40 * 1e3 / r["ms_per_step"] - r["value"]) / r["value"] < 1e-6


def test_fingerprint_ignores_comments_only():
    a = "int f(int x) {  // one\n  return x + 1; /* two\n lines */\n}\n"
    b = "int f(int x) {\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    files = ["k.cu"]
    h = lambda src: bench._sources_sha256(files, read=lambda rel: src)
    assert h(a) == h(b)
    assert h(b) != h(c)


@pytest.mark.parametrize("kernel", ["k_batched", "k_probe"])
def test_traffic_figure_only_for_the_captured_sources(kernel, monkeypatch):
    """The recorded DRAM bytes are reported (scaled by the documents of a
    launch) while the kernel's sources hash to the captured state, and null
    as soon as they do not."""
    t = bench._TRAFFIC[kernel]
    assert os.path.exists(os.path.join(ROOT, t["profile"]))
    for rel in t["sources"]:
        assert os.path.exists(os.path.join(ROOT, bench._CSRC, rel)), rel
    monkeypatch.setitem(bench._TRAFFIC, kernel,
                        dict(t, sha256=bench._sources_sha256(t["sources"])))
    assert bench._traffic(kernel, 1000) == pytest.approx(1000 * t["bytes_per_doc"])
    assert bench._traffic(kernel, 0) is None
    monkeypatch.setitem(bench._TRAFFIC, kernel, dict(t, sha256="0" * 64))
    assert bench._traffic(kernel, 1000) is None

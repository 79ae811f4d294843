"""CPU checks of bench.py's host logic: the roofline entry built from per-kernel times, the traffic
lookup keyed by the library source digest, the flop model, and the reference (oracle) arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1806_03095_gb300 import configs, roofline  # noqa: E402


def test_roofline_entry_takes_the_dominant_kernel():
    cfg = configs.WORKLOADS["tgv64_k3"](precision=0, kernel=2)
    kt = {"faces": (100.0, 10), "cell_stage": (120.0, 10), "dev": (1.0, 10)}
    r = bench.roofline_entry(kt, cfg, 0, {"hbm_gbs": 6000.0})
    Nc = 64 ** 3
    fl = roofline.kernel_flops("cell_stage", 4, 5, 4, Nc)
    assert r["kernel"] == bench.KERNEL_NAMES["cell_stage"]
    assert r["flops_per_launch"] == fl
    assert r["achieved"] == pytest.approx(fl / 12e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert set(r["kernels"]) == {"faces", "cell_stage", "dev"}
    assert sum(v["share"] for v in r["kernels"].values()) == pytest.approx(1.0, abs=1e-3)
    assert r["hbm"]["peak"] == 6000.0


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    key = ("faces", 0, 4, 5, 4)
    monkeypatch.setitem(bench.TRAFFIC, key, (1000.0, "digest-at-capture", "profiles/x.md"))
    monkeypatch.setattr(bench, "kernel_digest", lambda: "digest-at-capture")
    assert bench.traffic_per_launch("faces", 0, 4, 5, 4, 10) == (10000.0, "profiles/x.md")
    monkeypatch.setattr(bench, "kernel_digest", lambda: "another")
    t, src = bench.traffic_per_launch("faces", 0, 4, 5, 4, 10)
    assert t is None and "changed" in src
    assert bench.traffic_per_launch("faces", 1, 9, 13, 9, 10) == (None, None)  # never captured


@pytest.mark.parametrize("N,QC,QV", [(3, 4, 3), (4, 5, 4), (6, 8, 6)])
def test_face_centric_flops_below_element_centric(N, QC, QV):
    fc = 3 * roofline.face_pair_flops(N, QC, QV) + roofline.cell_stage_flops_per_cell(N, QC, QV)
    ec = roofline.stage_flops_per_cell(N, QC, QV)
    assert fc < ec
    # each face once for both cells costs less than each face twice
    assert 3 * roofline.face_pair_flops(N, QC, QV) < 6 * roofline.face_flops(N, QC, QV)


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_algorithmic_bytes_per_kernel_kind():
    """Per cell at k = 3 (320 values): the byte counts the roofline uses are the blocks each kernel moves.
    FP64: face kernel U + shares (2,560 + 7,680), cell + stage U, dU read and written, U_out, shares
    (4 x 2,560 + 7,680), split M^-1 + stage R, dU read and written, U, U_out (5 x 2,560).  Mixed form:
    the operator kernels read the FP32 deviation state and the stage kernels write the next one."""
    kb = lambda kind, rb: roofline.kernel_bytes(kind, 4, 1, rb)
    assert kb("faces", 8) == 2560 + 7680
    assert kb("cell_stage", 8) == 4 * 2560 + 7680
    assert kb("mass", 8) == 5 * 2560
    assert kb("fused", 8) == 4 * 2560
    assert kb("faces", 4) == 1280 + 3840
    assert kb("cell_stage", 4) == 2560 + 1280 + 2 * 1280 + 2560 + 1280 + 3840
    assert kb("mass", 4) == 1280 + 2 * 1280 + 2560 + 2560

"""Host logic of the bench line's profile-derived fields (no GPU): the pinned
ncu counters are used only for the code they were taken on, scaled per hit
from the captured batch to the measured one, and the issue roofline is the
scaled warp instructions over the live kernel time against 4 schedulers per
SM; without counters the roofline falls back to the HBM fraction."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// a kernel
__global__ void k(int* p) { /* body */ p[0] = 1; }
"""


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text(SRC)
    pin = {"source": "k.cu", "source_code_sha256": bench.code_digest(str(tmp_path / "k.cu")),
           "kernels": {"k<64>": {"dram_read_bytes": 300, "dram_write_bytes": 100, "hits": 1000,
                                 "warp_inst": 2_000_000, "thread_inst": 32_000_000}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(pin))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_digest_ignores_comments_and_whitespace(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(SRC)
    b.write_text("// another comment\n__global__   void k(int* p)\n{ p[0] = 1; }  /* x */\n")
    c.write_text(SRC.replace("p[0] = 1", "p[0] = 2"))
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_counters_only_for_the_captured_code_scaled_per_hit(fake_root):
    assert bench.profiled_traffic("k<64>", 1000) == 400
    assert bench.profiled_traffic("k<128>", 1000) is None      # another block size
    assert bench.profiled_traffic("k<64>", 5000) == pytest.approx(2000)   # per hit, a larger batch
    (fake_root / "k.cu").write_text(SRC.replace("p[0] = 1", "p[1] = 1"))
    assert bench.profiled_traffic("k<64>", 1000) is None       # the code changed


def test_issue_roofline_arithmetic(fake_root):
    r = bench.issue_roofline("k<64>", 1000, kernel_ms=1.0, sm_mhz=2000.0, sm_count=152)
    # 2e6 warp instructions in 1 ms = 2 G/s; peak 4 * 152 * 2.0 GHz = 1216 G/s
    assert r["achieved_ginst_s"] == pytest.approx(2.0)
    assert r["peak_ginst_s"] == pytest.approx(1216.0)
    assert r["frac"] == pytest.approx(2.0 / 1216.0)
    assert r["simt_efficiency"] == pytest.approx(0.5)
    assert bench.issue_roofline("k<64>", 1000, 1.0, None, 152) is None
    # a batch twice as large in the same time issues twice the instructions
    assert bench.issue_roofline("k<64>", 2000, 1.0, 2000.0, 152)["frac"] == pytest.approx(4.0 / 1216.0)


def test_roofline_entry_binds_on_issue_with_counters_else_hbm(fake_root):
    kms = [0.1, 1.0, 1.0, 0.1, 0.5]
    r = bench.roofline_entry(64, 1000, 100.0, 6000.0, "measured", kms, 2000.0, 152, 50.0, 20.0)
    # the search kernel's name is k_search_persistent<64>: no counters in the fake pin
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(100.0 / 6000.0) and r["traffic"] is None
    pin = json.loads((fake_root / "profiles" / "traffic.json").read_text())
    pin["kernels"]["k_search_persistent<64>"] = pin["kernels"]["k<64>"]
    (fake_root / "profiles" / "traffic.json").write_text(json.dumps(pin))
    r = bench.roofline_entry(64, 1000, 100.0, 6000.0, "measured", kms, 2000.0, 152, 50.0, 20.0)
    assert r["bound"] == "issue" and r["unit"] == "G warp instructions/s"
    assert r["frac"] == pytest.approx(2.0 / 1216.0) and r["hbm_frac"] == pytest.approx(100.0 / 6000.0)
    assert r["traffic"] == 400 and r["simt_efficiency"] == pytest.approx(0.5)


def test_a_step_of_several_kernels_sums_their_counters(fake_root):
    pin = json.loads((fake_root / "profiles" / "traffic.json").read_text())
    pin["kernels"]["k2"] = {"dram_read_bytes": 50, "dram_write_bytes": 50, "hits": 500,
                            "warp_inst": 1_000_000, "thread_inst": 8_000_000}
    (fake_root / "profiles" / "traffic.json").write_text(json.dumps(pin))
    # per hit: k<64> 0.4 B, k2 0.2 B; at 1000 hits 400 + 200
    assert bench.profiled_traffic(("k<64>", "k2"), 1000) == pytest.approx(600)
    r = bench.issue_roofline(("k<64>", "k2"), 1000, kernel_ms=1.0, sm_mhz=2000.0, sm_count=152)
    assert r["warp_inst"] == pytest.approx(4_000_000)
    assert r["simt_efficiency"] == pytest.approx((32e6 + 16e6) / (32 * 4e6))
    assert bench.profiled_traffic(("k<64>", "k3"), 1000) is None   # one of them has no counters

"""Host logic of the bench line's profile-derived fields (no GPU): the pinned
ncu counters are used only for the code they were taken on and only for the
batch they were taken on, and the issue roofline is the captured warp
instructions over the live kernel time against 4 schedulers per SM."""
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


def test_counters_only_for_the_captured_code_and_batch(fake_root):
    assert bench.profiled_traffic("k<64>", 1000) == 400
    assert bench.profiled_traffic("k<128>", 1000) is None      # another block size
    assert bench.profiled_traffic("k<64>", 999) is None        # another batch
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
    assert bench.issue_roofline("k<64>", 999, 1.0, 2000.0, 152) is None

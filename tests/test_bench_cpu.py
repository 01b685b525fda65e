"""Host logic of bench.py that needs no GPU: the committed ncu records it reads
(DRAM bytes, issue activity) parse, name existing sources, and are used only
while the source they were taken from is unchanged."""
import hashlib
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1611_01642_gb300", "csrc")


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _records(path):
    rec = {}
    for line in open(path):
        if line.startswith("@") and "=" in line:
            k, v = line[1:].split("=", 1)
            rec[k.strip()] = v.strip()
    return rec


def test_profile_records_are_well_formed():
    prof = os.path.join(ROOT, "profiles")
    names = sorted(os.listdir(prof))
    assert names and all(n.endswith((".txt", ".md")) for n in names)
    dram = _records(os.path.join(prof, "dram_per_kernel_1242x375_b64.txt"))
    assert {"k_resize", "k_cells", "k_svm_tc", "k_nms"} <= set(dram)
    for kernel, v in dram.items():
        src, h, nbytes = v.split()
        assert os.path.exists(os.path.join(CSRC, src)), kernel
        assert re.fullmatch(r"[0-9a-f]{16}", h), kernel
        assert float(nbytes) > 0, kernel
    for n in names:
        rec = _records(os.path.join(prof, n))
        if "source_sha256_16" in rec:
            assert re.fullmatch(r"[0-9a-f]{16}", rec["source_sha256_16"]), n
            for k, v in rec.items():
                if k != "source_sha256_16":
                    assert float(v) > 0, (n, k)


def _fake_tree(tmp_path, src_text):
    csrc = tmp_path / "paper_1611_01642_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_demo.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    return hashlib.sha256(src_text.encode()).hexdigest()[:16]


def test_recorded_figure_follows_the_source_hash(bench, tmp_path, monkeypatch):
    h = _fake_tree(tmp_path, "// kernel v1\n")
    (tmp_path / "profiles" / "k_demo.txt").write_text(
        f"summary\n@source_sha256_16 = {h}\n@dram_bytes_per_launch = 123000\n@issue_active_frac = 0.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k_demo.txt", "k_demo.cu") == 123000.0
    assert bench.recorded_traffic("k_demo.txt", "k_demo.cu", "issue_active_frac") == 0.5
    assert bench.recorded_traffic("k_demo.txt", "k_demo.cu", "missing_key") is None
    assert bench.recorded_traffic("absent.txt", "k_demo.cu") is None
    # the source changes: the figure no longer describes it
    (tmp_path / "paper_1611_01642_gb300" / "csrc" / "k_demo.cu").write_text("// kernel v2\n")
    assert bench.recorded_traffic("k_demo.txt", "k_demo.cu") is None


def test_hbm_per_kernel_scales_and_skips_changed_sources(bench, tmp_path, monkeypatch):
    h = _fake_tree(tmp_path, "// resize\n")
    (tmp_path / "profiles" / "dram_per_kernel_1242x375_b64.txt").write_text(
        f"@k_resize = k_demo.cu {h} 64000000\n@k_cells = k_demo.cu 0000000000000000 1000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 1000.0}, "measured"))
    out = bench.hbm_per_kernel([2.0, 1.0, 1.0, 1.0], "tc", 128)
    # 64 MB per 64 frames, 128 frames in 2 ms: 64 GB/s, 0.064 of a 1000 GB/s peak
    assert out["k_resize"]["dram_bytes"] == 128e6
    assert abs(out["k_resize"]["achieved_gbs"] - 64.0) < 1e-9
    assert abs(out["k_resize"]["frac_of_peak"] - 0.064) < 1e-12
    assert out["k_cells"] is None          # recorded for another source
    assert "k_svm_tc" not in out and "k_nms" not in out  # no record

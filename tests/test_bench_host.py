"""Host logic of bench.py that feeds the JSON line (no GPU): the DRAM-traffic
lookup behind roofline.traffic (per kernel and SpMM variant, scaled to the
workload, void once the kernel sources change) and the measured peaks."""
import os

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _kv(path):
    kv = {}
    with open(path) as f:
        for ln in f:
            if "=" in ln and not ln.startswith("#"):
                k, v = ln.split("=", 1)
                kv[k.strip()] = v.strip()
    return kv


def test_traffic_scales_by_units(bench, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    prof = os.path.join(bench.ROOT, "profiles")
    kv = _kv(os.path.join(prof, "fsai_tr_traffic.txt"))
    # (freshness is bench.py's runtime check: here the file's own hash stands in)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: kv["kernel_sha"])
    units = float(kv["units"])
    per = float(kv["dram_bytes_per_launch"])
    # scaled in proportion to the nonzeros of the timed workload
    assert bench.ncu_traffic("C5", "fsai_tr", units) == pytest.approx(per)
    assert bench.ncu_traffic("C5", "fsai_tr", 4 * units) == pytest.approx(4 * per)


def test_spmm_traffic_is_per_variant(bench, monkeypatch):
    prof = os.path.join(bench.ROOT, "profiles")
    sha = _kv(os.path.join(prof, "spmm_v1_traffic.txt"))["kernel_sha"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    for v in range(6):
        kv = _kv(os.path.join(prof, f"spmm_v{v}_traffic.txt"))
        assert kv["kernel_sha"] == sha  # one capture run for all variants
        assert kv["variant"] == str(v)
        got = bench.ncu_traffic("C5", "spmm", float(kv["units"]), v)
        assert got == pytest.approx(float(kv["dram_bytes_per_launch"]))
    # the stencil form (no column array) moves fewer bytes than the fixed-length one
    assert bench.ncu_traffic("C5", "spmm", 1.0, 5) < bench.ncu_traffic("C5", "spmm", 1.0, 1)
    # no capture for an unknown variant or kernel
    assert bench.ncu_traffic("C5", "spmm", 1.0, 9) is None
    assert bench.ncu_traffic("C5", "no_such_kernel", 1.0) is None


def test_stale_capture_reads_null(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "fsai_tr_traffic.txt").write_text("kernel_sha = 0000000000000000\nunits = 1\n"
                                              "dram_bytes_per_launch = 100\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "ffffffffffffffff")
    assert bench.ncu_traffic("C5", "fsai_tr", 1.0) is None
    (prof / "fsai_tr_traffic.txt").write_text("kernel_sha = ffffffffffffffff\nunits = 2\n"
                                              "dram_bytes_per_launch = 100\n")
    assert bench.ncu_traffic("C5", "fsai_tr", 1.0) == pytest.approx(50.0)


def test_measured_peaks_are_read(bench):
    pk = bench.measured_peaks()
    assert pk["hbm_gbs"] > 1000 and pk["source"] in ("measured", "fallback")

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


def test_l2_note_follows_the_working_set(bench):
    from synth import CONFIGS
    assert bench.stencil_size(2.0) == 12 and bench.stencil_size(3.0) == 28 and bench.stencil_size(1.0) == 4
    # the 2048^2 benchmark image and the batch outgrow the L2; the small images do not
    for name, big in (("C1", False), ("C2", False), ("C3", True), ("C5", True)):
        note = bench.workload_config(CONFIGS[name], 1)["l2"]
        assert ("inputs larger than L2" in note) == big, (name, note)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference on the small image: one JSON line with the
    oracle's timing, its CPU baseline and end-to-end objects."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(os.path.dirname(__file__)), "bench.py"),
                        "--impl", "reference", "--workload", "C1", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s/outer-iter" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["dtype"] == "f64" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("C1: 32x32")


def test_clock_samples_are_summarised(bench):
    """nvidia-smi lines (FIELDS order, csv, no units): median SM clock, the
    largest max clock, every reason active in any sample; unreadable lines
    are skipped and no readable sample gives None."""
    lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1100.2, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    out = bench.ClockSampler.summarise(lines)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = lines[:1] + ["0, 1500, 2070, 800, 0x40, Not Active, Active, Not Active, Not Active"]
    assert bench.ClockSampler.summarise(hot)["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler.summarise(["garbage"]) is None


def test_reference_arm_runs_on_rank_zero_only(bench, capsys):
    """Under torchrun the other ranks of the reference arm exit at once,
    without work or output."""
    import argparse
    args = argparse.Namespace(workload="C1", steps=1, warmup=1, gpus=2, cpu_window=192)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_computed_column_traffic_files(bench, monkeypatch):
    """The captures of the computed-column SpMM variants (6, 7) and of
    k_fsai_tr with computed columns (variant 1) come from one run; the
    computed-column SpMM moves fewer bytes per nonzero than the slot form."""
    prof = os.path.join(bench.ROOT, "profiles")
    kv6 = _kv(os.path.join(prof, "spmm_v6_traffic.txt"))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: kv6["kernel_sha"])
    for v in (6, 7):
        kv = _kv(os.path.join(prof, f"spmm_v{v}_traffic.txt"))
        assert kv["kernel_sha"] == kv6["kernel_sha"] and kv["variant"] == str(v)
        assert bench.ncu_traffic("C5", "spmm", float(kv["units"]), v) == pytest.approx(
            float(kv["dram_bytes_per_launch"]))
    kt = _kv(os.path.join(prof, "fsai_tr_v1_traffic.txt"))
    assert kt["kernel_sha"] == kv6["kernel_sha"] and kt["variant"] == "1"
    assert bench.ncu_traffic("C5", "fsai_tr", 2 * float(kt["units"]), 1) == pytest.approx(
        2 * float(kt["dram_bytes_per_launch"]))


def test_cpu_sample_direct_mode(bench):
    """The oracle's direct mode (sparse LU of A once, exact solves) beside its
    Jacobi-PCG mode on the 32x32 image (one window: the whole image): no PCG
    iterations and a factorisation time in the direct mode, PCG iterations
    and none in the other."""
    d = bench.run_cpu_sample("C1", 0.0, 1, 192, 12676, solver="direct")
    p = bench.run_cpu_sample("C1", 0.0, 1, 192, 12676)
    assert d["cores"] == 1 and d["scale"] == pytest.approx(1.0)
    assert d["iters"] == [0.0] and d["factor_s"] > 0.0
    assert p["iters"][0] > 0 and p["factor_s"] == 0.0

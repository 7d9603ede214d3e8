"""Host-side logic of bench.py, on the CPU: the DRAM traffic it reports is the
committed ncu figure only while that figure was taken on the current kernel
source, the clock summary reads nvidia-smi's CSV, and the HBM peak comes from
the measured file."""
import json
import os

import bench


def test_traffic_only_for_the_current_kernel(tmp_path, monkeypatch):
    b, e = bench.ncu_traffic("rmat22", "nb", 128)
    assert b is not None and b > 0 and e["kernel_sha"] == bench.kernel_hash()
    assert e["dram_bytes_read"] + e["dram_bytes_write"] == b
    assert bench.ncu_traffic("rmat22", "degree", 64) == (None, None)
    d = json.load(open(bench.TRAFFIC_FILE))
    for v in d.values():
        v["kernel_sha"] = "0" * 16
    stale = tmp_path / "traffic.json"
    stale.write_text(json.dumps(d))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(stale))
    assert bench.ncu_traffic("rmat22", "nb", 128) == (None, None)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.ncu_traffic("rmat22", "nb", 128) == (None, None)


def test_clock_summary(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()  # as if nvidia-smi had been started
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.proc = None
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_hbm_peak_is_the_measured_copy_bandwidth():
    peak, src = bench.hbm_peak()
    if os.path.exists(bench.PEAKS_FILE):
        assert src == "measured" and peak == float(json.load(open(bench.PEAKS_FILE))["hbm_gbs"])
    else:
        assert src == "fallback" and peak == 6800.0

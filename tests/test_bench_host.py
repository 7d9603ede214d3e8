"""Host-side logic of bench.py, on the CPU: the DRAM traffic it reports is the
committed ncu figure only while that figure was taken on the current kernel
source, the clock summary reads nvidia-smi's CSV, and the HBM peak comes from
the measured file."""
import json
import os

import bench


def test_traffic_only_for_the_current_kernel(tmp_path, monkeypatch):
    entry = {"kernel_sha": bench.kernel_hash(), "dram_bytes_read": 70, "dram_bytes_write": 30,
             "dram_bytes_per_step": 100}
    cur = tmp_path / "traffic.json"
    cur.write_text(json.dumps({"rmat22_nb_b128": entry}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(cur))
    b, e = bench.ncu_traffic("rmat22", "nb", 128)
    assert b == 100 and e["kernel_sha"] == bench.kernel_hash()
    assert bench.ncu_traffic("rmat22", "degree", 64) == (None, None)
    stale = tmp_path / "stale.json"
    stale.write_text(json.dumps({"rmat22_nb_b128": dict(entry, kernel_sha="0" * 16)}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(stale))
    assert bench.ncu_traffic("rmat22", "nb", 128) == (None, None)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.ncu_traffic("rmat22", "nb", 128) == (None, None)


def test_committed_traffic_entries_are_consistent():
    if not os.path.exists(bench.TRAFFIC_FILE):
        return
    for v in json.load(open(bench.TRAFFIC_FILE)).values():
        assert v["dram_bytes_read"] + v["dram_bytes_write"] == v["dram_bytes_per_step"]


def test_fixed_work_and_fixture_check():
    """The metric's fixed work is the oracle's plain NBCut arc count stored with
    the workload, and a result equal to the stored top-k passes the check
    while any change fails it (no GPU: results stand in as plain objects)."""
    from types import SimpleNamespace

    import numpy as np

    fx = bench.fixture_for("ba1m")
    if fx is None:
        return
    want = bench.fixture_results(fx, 10)[0]
    assert bench.plain_work(fx, 10) == want["oracle_counters"]["edges_visited"] > 0
    assert bench.plain_work(fx, 7) is None
    g = SimpleNamespace(offsets=np.zeros(1, np.uint32), cols=np.zeros(0, np.uint32))
    fx = dict(fx, graphs=[dict(fx["graphs"][0], csr_sha256=bench.csr_sha256(g))])
    res = SimpleNamespace(ids=np.array(want["ids"], np.uint32), dist_sum=np.array(want["S"], np.uint64),
                          reach=np.array(want["r"], np.uint32), n_tied_at_kth=want["n_tied"],
                          farness=np.array([float.fromhex(h) for h in want["farness_hex"]]))
    assert bench.matches_fixture([res], fx, 10, [g]) is True
    res.dist_sum = res.dist_sum.copy()
    res.dist_sum[3] += 1
    assert bench.matches_fixture([res], fx, 10, [g]) is False


def test_plan_bytes_formula():
    st = dict(n=100, batch_bits=128, row_bytes=16, td_levels=2, td_frontier=10, td_frontier_arcs=50,
              bu_levels=1, bu_scanned_vertices=30, bu_scanned_arcs=70)
    td = 10 * (8 + 16) + 4 * 50 + 2 * 16 * 50 + 3 * 16 * 100 * 2
    bu = 8 * 30 + (4 + 16) * 70 + 3 * 16 * 100 * 1
    assert bench.survey_level_bytes(st) == td + bu


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

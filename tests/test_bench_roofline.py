"""Host logic of bench.py's roofline line (no GPU): the achieved rate over the
busy time, the peak per kernel class, and the DRAM traffic taken from a
committed ncu summary only while its source hash matches."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

STATS = {"launches": 10, "flops": 1.0e12, "ms": 2000.0, "busy_ms": 1000.0}


def _write_profile(root, name, sha, traffic):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", f"{name}.md"), "w") as fh:
        fh.write(f"# x\n\ntraffic_bytes_per_full_launch: {traffic}\n\nsource_sha256: {sha}\n")


def test_traffic_is_read_by_workload_name_and_dropped_on_a_stale_hash(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha("history_fp64")  # the sources of the real tree
    monkeypatch.setattr(bench, "kernel_source_sha", lambda key: sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write_profile(tmp_path, "history_fp64_lorenz-single", sha, "5.25e6")
    line = bench.roofline("history", STATS, "fp64", {}, "lorenz-single")
    assert line["traffic"] == pytest.approx(5.25e6)
    _write_profile(tmp_path, "history_fp64_lorenz-single", "0" * 64, "5.25e6")
    assert bench.roofline("history", STATS, "fp64", {}, "lorenz-single")["traffic"] is None
    # no summary for another workload
    assert bench.roofline("history", STATS, "fp64", {}, "ml-scalar")["traffic"] is None


def test_achieved_uses_the_busy_time_and_the_class_peak():
    fp64 = bench.roofline("history", STATS, "fp64", {"sm_max_mhz": 2070.0}, "lorenz-single")
    assert fp64["bound"] == "alu" and fp64["unit"] == "GFLOP/s"
    assert fp64["achieved"] == pytest.approx(1.0e12 / 1.0 / 1e9)  # busy 1000 ms, not 2000
    assert fp64["peak"] == pytest.approx(4 * 152 * 2070e6 / 1e9)
    assert fp64["frac"] == pytest.approx(fp64["achieved"] / fp64["peak"])
    split = bench.roofline("history", STATS, "split", {"sm_max_mhz": 2070.0}, "duffing-sweep")
    assert split["bound"] == "tensor" and split["unit"] == "TFLOP/s"
    assert split["achieved"] == pytest.approx(6 * 1.0e12 / 1.0 / 1e12)  # 6 bf16 products
    x2 = bench.roofline("history", STATS, "fp64x2", {"sm_max_mhz": 2070.0}, "lorenz-single")
    assert "double-double" in x2["peak_note"]


def test_committed_summaries_name_their_command_and_hash():
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert "ncu " in txt and "--clock-control none" in txt, name
        assert "source_sha256:" in txt and "traffic_bytes_per_full_launch:" in txt, name


def test_headline_is_the_solve_work_over_the_uninstrumented_step():
    """With the workload and the uninstrumented step time given, `achieved` is
    2 N^2 flops per column (x6 bf16 products on the tensor path) over
    ms_per_step, and the instrumented per-launch rate moves to `in_launch`."""
    import fabm_workloads as wl
    w = wl.lorenz_long(B=4, N=1024)
    macs = w.history_macs()
    assert macs == pytest.approx(4 * 3 * 1024.0 ** 2)
    line = bench.roofline("history", STATS, "split", {"sm_max_mhz": 2070.0}, "lorenz-long",
                          w, 100.0)
    assert line["achieved"] == pytest.approx(6 * 2 * macs / 0.1 / 1e12)
    assert line["work_per_step"] == pytest.approx(6 * 2 * macs)
    assert line["in_launch"]["achieved"] == pytest.approx(6 * 1.0e12 / 1.0 / 1e12)
    assert line["frac"] == pytest.approx(line["achieved"] / line["peak"])
    fp64 = bench.roofline("history", STATS, "fp64", {"sm_max_mhz": 2070.0}, "lorenz-single",
                          w, 100.0)
    assert fp64["achieved"] == pytest.approx(2 * macs / 0.1 / 1e9)


def test_dtype_names_every_history_kernel():
    """The bench line's dtype comes from the kernel a solve ran: every history
    kernel name of the binding maps to the arithmetic it computes in."""
    import paper_1710_01133_gb300 as fabm
    assert set(bench.DTYPE_OF_HISTORY) == set(fabm.HIST) - {"auto"}
    assert bench.DTYPE_OF_HISTORY["tensor-wide"] == "bf16x3"
    assert bench.DTYPE_OF_HISTORY["fp32c"] == "f32c"
    assert bench.DTYPE_OF_HISTORY["x2"] == "f64x2"

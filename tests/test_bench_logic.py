"""Host-side arithmetic of bench.py's JSON line, on synthetic kernel statistics: the roofline
entries (achieved = algorithmic work / event-timed device time, frac = achieved / peak, the
family with the larger device time as the line's roofline) and the whole-job rate of replicas."""

import os
import sys

import pytest

pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _Args:
    precision = "mixed"
    workload = "const2d_640"


def test_roofline_entries_and_main_family():
    # two DDM applications profiled: substitutions 2.9 ms over 4 launches, trace 2.75 ms over 2
    stats = {"subst": (4, 2.9), "trace_step": (2, 2.75), "assemble": (4, 0.36), "extract": (4, 0.14),
             "krylov": (10, 3.0)}
    work = (18.4e9 * 2, 11.3e9)          # per DDM application: 2 substitution launches, 1 trace
    geo = {"plan": 2, "nrhs": 16, "nsub": 64, "T": 832, "Nglob": 664 * 664, "Nloc": 104 * 104,
           "sweeps": 8, "panel_width": 16, "panels_per_cta": 1}
    main, entries = bench.roofline_entry(stats, work, 2, _Args(), geo)
    by = {e["kernel"].split(" ")[0]: e for e in entries}
    sub = by["k_subst_tc<tf32>"]
    assert sub["bound"] == "tensor" and sub["unit"] == "TFLOP/s"
    assert sub["achieved"] == pytest.approx(18.4e9 * 2 * 2 / 2.9e-3 / 1e12)
    assert sub["frac"] == pytest.approx(sub["achieved"] / sub["peak"])
    assert sub["avg_launch_ms"] == pytest.approx(2.9 / 4)
    # no counters of the substitution kernel as it stands were taken on this workload
    assert sub["traffic"] is None
    tr = by["k_trace_sweeps<float>"]
    assert tr["bound"] == "alu"
    assert tr["achieved"] == pytest.approx(11.3e9 * 2 / 2.75e-3 / 1e12)
    asm = by["k_assemble"]
    assert asm["bound"] == "hbm" and asm["unit"] == "GB/s"
    assert asm["achieved"] == pytest.approx(asm["bytes_per_launch"] * 2 * 2 / 0.36e-3 / 1e9)
    # no DRAM counters were taken for this workload's HBM kernels
    assert asm["traffic"] is None
    # the family with the larger device time carries the line
    assert main["kernel"] == sub["kernel"] and "family_share" in main


def test_whole_job_rate_of_replicas():
    assert bench.whole_job_rate(1, 16, 5, 0.025) == pytest.approx(3200.0)
    assert bench.whole_job_rate(4, 16, 5, 0.025) == pytest.approx(4 * 3200.0)
    assert bench.whole_job_rate(2, 16, 5, 0.0) is None


def test_roofline_traffic_follows_the_launch_shape():
    """DRAM bytes are attached only to the workload and launch shape they were counted on."""
    stats = {"subst": (6, 16.0), "trace_step": (3, 9.3), "assemble": (6, 4.6), "extract": (6, 1.8)}
    work = (2 * 178.6e9, 202e9)
    geo = {"plan": 2, "nrhs": 64, "nsub": 256, "T": 704, "Nglob": 1048 * 1048, "Nloc": 88 * 88,
           "sweeps": 8, "trace_kernel": 0, "panel_width": 16, "panels_per_cta": 2}

    class A(_Args):
        workload = "layer2d_1024"

    _, entries = bench.roofline_entry(stats, work, 3, A(), geo)
    by = {e["kernel"].split(" ")[0]: e for e in entries}
    assert by["k_subst_tc<tf32>"]["traffic"] == bench.SUBST_TRAFFIC[("mixed", "layer2d_1024", 16, 2)]
    assert by["k_trace_tc<tf32>"]["traffic"] == bench.TRACE_TC_TRAFFIC[("mixed", "layer2d_1024")]
    assert by["k_assemble"]["traffic"] == bench.HBM_TRAFFIC[("mixed", "layer2d_1024")]["assemble"] / 2
    _, entries = bench.roofline_entry(stats, work, 3, A(), dict(geo, panel_width=32, panels_per_cta=1))
    by = {e["kernel"].split(" ")[0]: e for e in entries}
    assert by["k_subst_tc<tf32>"]["traffic"] is None


def test_tensor_entries_report_the_measured_mma_rate():
    """With the measured dense rate of the piece type, each tensor entry also gives its fraction of
    a third of it (three split products per useful product); other entries are unchanged."""
    stats = {"subst": (6, 16.0), "trace_step": (3, 9.3), "assemble": (6, 4.6), "extract": (6, 1.8)}
    work = (2 * 178.6e9, 202e9)
    geo = {"plan": 2, "nrhs": 64, "nsub": 256, "T": 704, "Nglob": 1048 * 1048, "Nloc": 88 * 88,
           "sweeps": 8, "trace_kernel": 0, "panel_width": 16, "panels_per_cta": 2}
    _, entries = bench.roofline_entry(stats, work, 3, _Args(), geo, mma_rate=1209.0)
    by = {e["kernel"].split(" ")[0]: e for e in entries}
    for k in ("k_subst_tc<tf32>", "k_trace_tc<tf32>"):
        assert by[k]["mma_rate_peak"] == pytest.approx(403.0)
        assert by[k]["frac_of_mma_rate"] == pytest.approx(by[k]["achieved"] / 403.0)
    assert "frac_of_mma_rate" not in by["k_assemble"]

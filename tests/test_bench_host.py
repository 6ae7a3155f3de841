"""Host-side bookkeeping of bench.py: the roofline object (the DRAM-traffic
lookup keyed by the CUDA sources' hash, the choice of the dominant Legendre
kernel, achieved / peak) and the clock summary of the timed region.  No GPU:
the plan is a stand-in that answers the few size queries the roofline needs,
and the clock samples are written in nvidia-smi's CSV form."""
import hashlib
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tree(tmp_path, sources):
    src = tmp_path / "paper_2510_01785_gb300" / "csrc"
    src.mkdir(parents=True)
    for name, text in sources.items():
        (src / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256()
    for name in sorted(sources):
        if name.endswith((".cu", ".cuh")):
            h.update(sources[name].encode())
    return h.hexdigest()[:16]


def test_kernel_traffic_matches_source_hash(tmp_path, monkeypatch):
    sha = _tree(tmp_path, {"a.cu": "x", "b.cuh": "y", "notes.txt": "ignored"})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k_legendre_tc<analysis>") is None  # no summary file
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# comment line\n"
        f"kernel=k_legendre_tc<analysis> source_sha={sha} dram_bytes_per_launch=123.5 scale=2\n"
        "kernel=k_legendre_tc<synthesis> source_sha=0000000000000000 dram_bytes_per_launch=7\n")
    assert bench.kernel_traffic("k_legendre_tc<analysis>") == 123.5
    # captured from another source: stale, so no figure
    assert bench.kernel_traffic("k_legendre_tc<synthesis>") is None
    assert bench.kernel_traffic("k_unknown") is None
    # a change to any .cu/.cuh file makes every line stale; other files do not count
    (tmp_path / "paper_2510_01785_gb300" / "csrc" / "notes.txt").write_text("changed")
    assert bench.kernel_traffic("k_legendre_tc<analysis>") == 123.5
    (tmp_path / "paper_2510_01785_gb300" / "csrc" / "b.cuh").write_text("y2")
    assert bench.kernel_traffic("k_legendre_tc<analysis>") is None


def test_committed_traffic_lines_are_well_formed():
    """Each line of the committed summary names a kernel, the source hash it
    was captured from and bytes per launch; the measured traffic stays near
    the algorithmic bytes (no wasted re-reads) for the table kernels."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        pytest.skip("no traffic summary committed")
    lines = [ln for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert lines
    for ln in lines:
        kv = dict(p.split("=", 1) for p in ln.split() if "=" in p)
        assert kv["kernel"].startswith("k_")
        assert len(kv["source_sha"]) == 16
        int(kv["source_sha"], 16)
        assert float(kv["dram_bytes_per_launch"]) > 0
        if "ratio" in kv:
            assert 0.8 < float(kv["ratio"]) < 1.25


class _Plan:
    """Stand-in for a plan at the bench workload."""

    def __init__(self):
        self.nalm = (bench.MMAX + 1) * (bench.LMAX + 1) - bench.MMAX * (bench.MMAX + 1) // 2
        self.table_bytes = 30_000_000_000
        self.column_table_bytes = 31_000_000_000
        self.nbatch = bench.NBATCH

    def chain_stats(self):
        return 4_000_000_000, 5_000_000_000


def _stages(ana_ms, syn_ms, tc):
    s = {"legendre_analysis": {"ms_per_step": ana_ms, "ms_per_launch": ana_ms, "launches": 1},
         "legendre_synthesis": {"ms_per_step": syn_ms, "ms_per_launch": syn_ms, "launches": 1},
         "ring_fft_analysis": {"ms_per_step": 0.5, "ms_per_launch": 0.5, "launches": 1},
         "ring_fft_synthesis": {"ms_per_step": 1.0, "ms_per_launch": 1.0, "launches": 1}}
    if tc:
        s["analysis_operand_pack"] = {"ms_per_step": 0.3, "ms_per_launch": 0.3, "launches": 1}
    return s


def test_table_roofline_takes_the_slower_kernel(monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda k: None)
    plan = _Plan()
    st = _stages(4.0, 5.0, tc=True)
    r = bench.legendre_roofline(plan, st, table=True)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["kernel"] == "k_legendre_tc<synthesis>"
    assert r["achieved"] == st["legendre_synthesis"]["hbm_gbs_algorithmic"]
    assert r["frac"] == pytest.approx(r["achieved"] / bench.HBM_PEAK_GBS)
    # the tensor-core synthesis streams the column copy of the table
    assert r["achieved"] > plan.column_table_bytes / 5e-3 / 1e9
    assert r["achieved"] < 1.1 * plan.column_table_bytes / 5e-3 / 1e9
    # the analysis streams the row table: slower stage flips the choice
    st = _stages(6.0, 5.0, tc=True)
    r = bench.legendre_roofline(plan, st, table=True)
    assert r["kernel"] == "k_legendre_tc<analysis>"
    assert plan.table_bytes / 6e-3 / 1e9 < r["achieved"] < 1.1 * plan.table_bytes / 6e-3 / 1e9
    # every FFT stage and the pack get an algorithmic bandwidth
    for k in ("ring_fft_analysis", "ring_fft_synthesis", "analysis_operand_pack"):
        assert st[k]["hbm_gbs_algorithmic"] > 0
    # the analysis ring FFT moves the maps and the spectra once each
    map_b = 4 * bench.NBATCH * 12 * bench.NSIDE ** 2
    spec_b = 8 * bench.NBATCH * (6 * bench.NSIDE ** 2 + 4 * bench.NSIDE - 1)
    assert st["ring_fft_analysis"]["hbm_gbs_algorithmic"] == pytest.approx((map_b + spec_b) / 0.5e-3 / 1e9)


def test_cuda_core_table_and_recompute_rooflines(monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda k: None)
    plan = _Plan()
    r = bench.legendre_roofline(plan, _stages(6.0, 5.0, tc=False), table=True)
    assert r["kernel"] == "k_legendre_analysis<table>" and r["bound"] == "hbm"
    st = _stages(40.0, 50.0, tc=False)
    r = bench.legendre_roofline(plan, st, table=False)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["kernel"] == "k_legendre_synthesis"
    active, _ = plan.chain_stats()
    # 3 FP64 flop per significant triple over the launch
    assert r["achieved"] == pytest.approx(3.0 * active / 50e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert "hbm_gbs_algorithmic" not in st["legendre_synthesis"]


def _smi_line(t, sm, reasons=()):
    """One nvidia-smi CSV line in the sampler's field order."""
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int(round((t % 1) * 1000) % 1000)
    flags = ["Active" if n in reasons else "Not Active"
             for n in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join([stamp, "0", str(sm), "2070", "900.00", "0x0"] + flags)


def test_clock_summary_keeps_the_timed_region():
    t0 = 1_900_000_000.0
    lines = [_smi_line(t0 - 1.0, 1200, ["sw_thermal_slowdown"]),  # before the region
             _smi_line(t0 + 0.10, 2070), _smi_line(t0 + 0.15, 2055, ["sw_power_cap"]),
             _smi_line(t0 + 0.20, 2070),
             _smi_line(t0 + 2.0, 600)]                               # after it (idle)
    r = bench.summarize_clocks("\n".join(lines), t0, t0 + 0.25)
    assert r["in_region"] and r["samples"] == 3
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]  # the thermal flag before the region does not count


def test_clock_summary_falls_back_to_all_samples():
    t0 = 1_900_000_000.0
    lines = [_smi_line(t0 + 1.0, 2070), _smi_line(t0 + 1.05, 2060, ["hw_slowdown"]), "garbage", ""]
    r = bench.summarize_clocks("\n".join(lines), t0, t0 + 0.01)
    assert not r["in_region"] and r["samples"] == 2
    assert r["sm_mhz"] == 2065 and r["reasons"] == ["hw_slowdown"]
    assert bench.summarize_clocks("", t0, t0 + 1)["sm_mhz"] is None


def test_oracle_legs_use_the_host_cores(monkeypatch):
    """The oracle timing runs alone on rank 0: it takes every core the
    process may use, whatever OMP_NUM_THREADS torchrun set for the ranks."""
    monkeypatch.setenv("OMP_NUM_THREADS", "1")
    n = bench.host_cores()
    assert 1 <= n <= (os.cpu_count() or 1)

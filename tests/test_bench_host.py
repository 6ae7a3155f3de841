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
    """A stand-in source tree; returns the hash of the tile kernels' sources
    (hpx_tc.cu, hpx_internal.cuh, include/hpx.h, in that order)."""
    src = tmp_path / "paper_2510_01785_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    for name, text in sources.items():
        (tmp_path / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256()
    for name in ("paper_2510_01785_gb300/csrc/hpx_tc.cu", "paper_2510_01785_gb300/csrc/hpx_internal.cuh",
                 "include/hpx.h"):
        h.update(sources[name].encode())
    return h.hexdigest()[:16]


def test_kernel_traffic_matches_source_hash(tmp_path, monkeypatch):
    C = "paper_2510_01785_gb300/csrc/"
    sha = _tree(tmp_path, {C + "hpx_tc.cu": "x", C + "hpx_internal.cuh": "y", "include/hpx.h": "z",
                           C + "hpx_fft.cu": "w"})
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
    # a change to a source the tiles are not built from does not count; one
    # to any of theirs makes every line stale
    (tmp_path / C / "hpx_fft.cu").write_text("changed")
    assert bench.kernel_traffic("k_legendre_tc<analysis>") == 123.5
    (tmp_path / C / "hpx_internal.cuh").write_text("y2")
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


def _bytes():
    nalm = _Plan().nalm
    return {"map": 4 * bench.NBATCH * 12 * bench.NSIDE ** 2, "alm": 8 * bench.NBATCH * nalm,
            "spec": 8 * bench.NBATCH * (6 * bench.NSIDE ** 2 + 4 * bench.NSIDE - 1),
            "F": 8 * bench.NBATCH * (4 * bench.NSIDE - 1) * (bench.MMAX + 1)}


def test_table_roofline_takes_the_slower_kernel(monkeypatch):
    """Algorithmic bytes: 4 B per significant lambda plus the stage's own
    input and output; the table's padding (table_bytes) does not count."""
    monkeypatch.setattr(bench, "kernel_traffic", lambda k: None)
    plan = _Plan()
    active, _ = plan.chain_stats()
    b = _bytes()
    st = _stages(4.0, 5.0, tc=True)
    r = bench.legendre_roofline(plan, st, table=True)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["kernel"] == "k_legendre_tc<synthesis>"
    assert r["achieved"] == st["legendre_synthesis"]["hbm_gbs_algorithmic"]
    assert r["frac"] == pytest.approx(r["achieved"] / bench.HBM_PEAK_GBS)
    assert r["achieved"] == pytest.approx((4 * active + b["alm"] + b["F"]) / 5e-3 / 1e9)
    assert r["algorithmic_bytes"] == 4 * active + b["alm"] + b["F"]
    # the slower stage flips the choice; the analysis reads spectra, writes alm
    st = _stages(6.0, 5.0, tc=True)
    r = bench.legendre_roofline(plan, st, table=True)
    assert r["kernel"] == "k_legendre_tc<analysis>"
    assert r["achieved"] == pytest.approx((4 * active + b["spec"] + b["alm"]) / 6e-3 / 1e9)
    # 16-bit single-part tables: 2 B per value
    r2 = bench.legendre_roofline(plan, _stages(6.0, 5.0, tc=True), table=True, value_bytes=2)
    assert r2["achieved"] == pytest.approx((2 * active + b["spec"] + b["alm"]) / 6e-3 / 1e9)
    # every FFT stage and the pack get an algorithmic bandwidth
    for k in ("ring_fft_analysis", "ring_fft_synthesis", "analysis_operand_pack"):
        assert st[k]["hbm_gbs_algorithmic"] > 0
    # the analysis ring FFT moves the maps and the spectra once each
    assert st["ring_fft_analysis"]["hbm_gbs_algorithmic"] == pytest.approx((b["map"] + b["spec"]) / 0.5e-3 / 1e9)
    assert st["ring_fft_synthesis"]["hbm_gbs_algorithmic"] == pytest.approx((b["F"] + b["map"]) / 1.0e-3 / 1e9)


def test_cuda_core_table_and_recompute_rooflines(monkeypatch):
    monkeypatch.setattr(bench, "kernel_traffic", lambda k: None)
    plan = _Plan()
    # a stage that ran no launch in the timed region gets no bandwidth
    st = _stages(6.0, 5.0, tc=False)
    st["synthesis_operand_pack"] = {"ms_per_step": 0.0, "ms_per_launch": 0.0, "launches": 0}
    bench.legendre_roofline(plan, st, table=False)
    assert "hbm_gbs_algorithmic" not in st["synthesis_operand_pack"]
    r = bench.legendre_roofline(plan, _stages(6.0, 5.0, tc=False), table=True)
    assert r["kernel"] == "k_legendre_analysis<table>" and r["bound"] == "hbm"
    st = _stages(40.0, 50.0, tc=False)
    r = bench.legendre_roofline(plan, st, table=False)
    assert r["bound"] == "alu" and r["unit"] == "TOP/s"
    assert r["kernel"] == "k_legendre_synthesis"
    active, _ = plan.chain_stats()
    # a double-FP32 step (19 FP32 operations) and 2 FMA per channel per significant triple
    assert r["achieved"] == pytest.approx((19 + 2 * bench.NBATCH) * active / 50e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_OPS_PEAK)
    assert "hbm_gbs_algorithmic" not in st["legendre_synthesis"]


def _full_line():
    """A record shaped like the benchmark's, with its bulky sub-records."""
    big = {"stages": {f"s{i}": {"ms_per_step": 1.234567, "launches": 3} for i in range(20)},
           "sample": list(range(64))}
    return {"metric": bench.METRIC, "value": 712.123456789, "unit": bench.UNIT, "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 11.2345678, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "precision": "FP32 I/O; FP64 lambda; FP16 hi/lo products",
            "data": "synthetic", "config": bench.workload_config(1),
            "roofline": {"bound": "hbm", "kernel": "k_legendre_tc<synthesis>", "achieved": 6345.6789,
                         "peak": 6791.0, "unit": "GB/s", "frac": 0.9344, "traffic": 2.9e10,
                         "peak_source": "measured", "work": "x" * 300, "algorithmic_bytes": 29890000000},
            "cpu_baseline": {"value": 0.021, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                             "sample": "oracle tier B (FP64 C, OpenMP): 64 of 3072 m columns analysed and 64 "
                                       "of 4095 rings synthesised, 8 ch; extrapolated x48 and x64",
                             "seconds": 7.1},
            "e2e": {"value": 678.9, "unit": bench.UNIT, "h2d_bytes_per_step": 704_643_072,
                    "d2h_bytes_per_step": 704_643_072, "calls": "y" * 200, "blocking_calls_value": 400.0},
            "gpu_launches": 180, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 7,
                                            "in_region": True, "reasons": []},
            "serving": big, "mixed_precision": big, "next_rows": big, "out_of_core": big, "other_configs": big,
            "cuda_core_table": big, "lambda_recompute": big, "tensor_core_tf32x3": big}


def test_headline_is_short_and_complete():
    """The line printed last fits in the 1.5 KB a driver keeps of stdout and
    carries the contract's keys; the bulky sub-records stay in the file."""
    import json
    line = _full_line()
    assert len(json.dumps(line)) > 4000
    h = bench.headline(line, "gpurun_out/bench_record.json")
    text = json.dumps(h)
    assert len(text) < 1500, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in h, k
    assert set(h["roofline"]) == {"bound", "kernel", "achieved", "peak", "unit", "frac", "traffic"}
    assert set(h["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert h["value"] == pytest.approx(line["value"], rel=1e-4)
    assert h["config"]["workload"] == bench.WORKLOAD
    for k in ("serving", "mixed_precision", "stages", "next_rows"):
        assert k not in h


def test_emit_writes_the_record_and_prints_one_line(tmp_path, capsys):
    import json
    line = _full_line()
    path = str(tmp_path / "out" / "rec.json")
    bench.emit(line, path)
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    h = json.loads(out[0])
    assert h["record"] == path and h["value"] == pytest.approx(712.123, rel=1e-6)
    assert json.load(open(path)) == json.loads(json.dumps(line))


def test_reference_arm_times_what_it_measured(tmp_path, monkeypatch, capsys):
    """The oracle arm: ms_per_step is the measured time of each sampled step
    (so ms_per_step x steps is the timed region), and value is the sampled
    work in full-step pairs over that time; the two arms share config."""
    import json
    pytest.importorskip("oracle")
    monkeypatch.setattr(bench, "NSIDE", 8)
    monkeypatch.setattr(bench, "LMAX", 23)
    monkeypatch.setattr(bench, "MMAX", 23)
    monkeypatch.setattr(bench, "NBATCH", 2)
    monkeypatch.setattr(bench, "WORKLOAD", "healpix-sht-nside8-lmax23-b2-f32")
    args = type("A", (), {"steps": 2, "warmup": 1, "record": str(tmp_path / "rec.json")})()
    t0 = time.perf_counter()
    assert bench.run_reference(args) == 0
    wall = time.perf_counter() - t0
    h = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert h["impl"] == "reference" and h["steps"] == 2 and h["warmup"] == 1
    assert h["ms_per_step"] * h["steps"] / 1e3 <= wall
    rec = json.load(open(str(tmp_path / "rec_reference.json")))
    assert 0 < rec["sample_fraction_of_step"] <= 1
    assert rec["extrapolated_ms_per_full_step"] >= rec["ms_per_step"]
    # value = sampled share of a step x channels / measured seconds
    assert h["value"] == pytest.approx(2 * rec["sample_fraction_of_step"] / (rec["ms_per_step"] / 1e3),
                                       rel=1e-3)
    assert h["config"] == bench.workload_config(1)
    assert h["e2e"]["h2d_bytes_per_step"] == 0


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

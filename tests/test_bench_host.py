"""CPU: the benchmark's host logic (clock samples, the committed DRAM traffic
keyed by kernel source, the peak file, algorithmic bytes per phase) and the
summary of a per-halo trace."""
import json
import os
import shutil
import types

import numpy as np
import pytest

import bench


def test_clock_summary_median_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1375.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1201.9, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2040.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3
    s.lines = ["0, 1500, 2070, 900, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() is None


def _tree(tmp_path):
    """A copy of the kernel sources the traffic entries are keyed on."""
    for files in bench.PHASE_SOURCES.values():
        for f in files:
            dst = tmp_path / f
            dst.parent.mkdir(parents=True, exist_ok=True)
            shutil.copyfile(os.path.join(bench.ROOT, f), dst)
    (tmp_path / "profiles").mkdir(exist_ok=True)


def test_measured_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(7, "batch") is None            # no summary at all
    entry = {"kernel": "cluster16_128k", "dram_bytes_per_launch": 1234.0, "launches": 3,
             "source_hash": bench.source_hash(bench.PHASE_SOURCES[7])}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"batch:7": entry}))
    assert bench.measured_traffic(7, "batch") == 1234.0
    assert bench.measured_traffic(0, "batch") is None            # no entry for that phase
    assert bench.measured_traffic(7, "sweep") is None            # nor for that workload
    # an edit of a kernel source the entry was measured on voids it
    with open(tmp_path / bench.PHASE_SOURCES[7][0], "a") as f:
        f.write("\n// edited\n")
    assert bench.measured_traffic(7, "batch") is None


def test_source_hash_depends_on_every_file(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    files = bench.PHASE_SOURCES[0]
    h0 = bench.source_hash(files)
    assert h0 == bench.source_hash(list(files))
    with open(tmp_path / files[-1], "a") as f:
        f.write(" ")
    assert bench.source_hash(files) != h0


def test_peaks_measured_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7012.5}))
    assert bench.peaks() == (7012.5, "measured")


def test_phase_bytes_of_a_small_batch():
    # two on-chip haloes (warp class, 8k class) and one multi-CTA halo;
    # float32 coordinates with per-particle masses: 7 x 4 B per candidate
    pop = types.SimpleNamespace(coord_type=1, m=np.ones(1), count=np.array([300, 6000, 200_000]))
    res = {"n_bound": np.array([250, 5000, 150_000]), "n_member": np.array([280, 5600, 180_000]),
           "part_iter": np.array([560, 16_800, 720_000])}
    cls = np.array([0, 3, 8])
    out = bench.phase_bytes(pop, res, cls)
    assert out.shape == (12,)
    assert out[0] == 28 * 300 + 12 * 250 + 88
    assert out[3] == 28 * 6000 + 12 * 5000 + 88
    assert out[1] == out[2] == out[4] == out[5] == out[6] == out[7] == 0
    # multi-CTA class: the radial stream (w.x, w.y, w.z, r) + m, 20 B per member
    assert out[8] == 28 * 200_000 + 20 * 180_000
    assert out[9] == 20 * 720_000
    assert out[10] == 20 * 180_000 + 12 * 150_000 + 88 + 32 * bench.N_BINS
    assert out[11] == (16 + 8) * (250 + 5000 + 150_000) + 32 * bench.N_BINS * 3
    # float64 coordinates, uniform mass: 6 x 8 B per candidate
    pop64 = types.SimpleNamespace(coord_type=0, m=None, count=pop.count)
    assert bench.phase_bytes(pop64, res, cls)[0] == 48 * 300 + 12 * 250 + 88


def test_trace_summary_of_a_synthetic_trace():
    from paper_0904_3662_gb300 import ahf, trace_report
    # rows: start, gathered, sorted, filled, iterated, done (ns), SM, variant + 256 * iterations
    t = np.array([
        [1000, 2000, 4000, 5000, 9000, 11000, 3, 0 + 256 * 2],     # warp class, 2 iterations
        [3000, 3500, 6500, 7000, 12000, 15000, 4, 0 + 256 * 4],    # warp class, 4 iterations
        [500, 1500, 3500, 4500, 8500, 10500, 7, 7 + 256 * 6],      # 16-CTA cluster
        [0, 0, 0, 0, 0, 0, 0, 0],                                  # not an on-chip halo: left out
    ], dtype=np.int64)
    s = trace_report.summarize(t)
    assert s["haloes"] == 3
    assert s["span_us"] == (15000 - 500) / 1e3
    w = s["variants"][ahf.PHASE_NAMES[0]]
    assert w["haloes"] == 2 and w["iterations_mean"] == 3.0
    assert w["first_start_us"] == 0.5 and w["last_end_us"] == 14.5
    assert w["gather_us_mean"] == 0.75 and w["sort_us_mean"] == 2.5 and w["fill_us_mean"] == 0.75
    assert w["iterate_us_mean"] == 4.5 and w["emit_us_mean"] == 2.5
    assert w["halo_us_mean"] == 11.0 and w["halo_us_max"] == 12.0
    c = s["variants"][ahf.PHASE_NAMES[7]]
    assert c["haloes"] == 1 and c["iterations_mean"] == 6.0 and c["first_start_us"] == 0.0
    tab = trace_report.table(s).splitlines()
    assert len(tab) == 2 + 2 and tab[2].startswith(f"| {ahf.PHASE_NAMES[0]} | 2 | 3.0 |")
    assert trace_report.summarize(np.zeros((4, 8), dtype=np.int64)) == {"haloes": 0}


def test_issue_roofline_counts_issue_slots():
    e = {"warp_instructions_per_launch": 4 * 152 * 2070e6 * 1e-3 * 0.25}   # a quarter of 1 ms of slots
    r = bench.issue_roofline(e, 1.0, 2070.0, 152)
    assert abs(r["frac"] - 0.25) < 1e-12
    assert bench.issue_roofline({"warp_instructions_per_launch": None}, 1.0, 2070.0, 152) is None
    assert bench.issue_roofline(None, 1.0, 2070.0, 152) is None


def test_ncu_launch_list_to_phases(tmp_path):
    from paper_0904_3662_gb300 import ncu_traffic as nt
    assert nt.phase_of("void warp_kernel<1>(OnchipLaunch)") == 0
    assert nt.phase_of("void unbind_kernel<512, 8192, 1, 16>(OnchipLaunch)") == 7
    assert nt.phase_of("void unbind_kernel<256, 4096, 1, 1>(OnchipLaunch)") == 2
    assert nt.phase_of("void unnamed>::g_halo<float, 1, 1024>(GridLaunch, int)") == 8
    assert nt.phase_of("void unnamed>::g_halo<float, 0, 256>(GridLaunch, int)") == 9
    assert nt.phase_of("unnamed>::g_pass_tma(GridLaunch, int)") == 9
    assert nt.phase_of("void unnamed>::g_rows_mixed(GridLaunch)") == 10
    assert nt.phase_of("void at::native::FillFunctor<float>") is None
    head = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = []
    launches = [("void unnamed>::g_scales<float>(GridLaunch)", 1000, 10, 5),
                ("void unnamed>::g_scatter<unsigned int, float, 0, 1>(GridLaunch)", 2000, 100, 7),
                ("unnamed>::g_pass_tma(GridLaunch, int)", 3000, 50, 11),
                ("unnamed>::g_pass_tma(GridLaunch, int)", 3000, 50, 11),
                ("void warp_kernel<1>(OnchipLaunch)", 500, 8, 3),
                ("void warp_kernel<1>(OnchipLaunch)", 700, 12, 5)]
    for i, (k, ns, mb, minst) in enumerate(launches):
        rows.append(f'"{i}","{k}","gpu__time_duration.sum","usecond","{ns / 1e3}"')
        rows.append(f'"{i}","{k}","dram__bytes_read.sum","Mbyte","{mb}"')
        rows.append(f'"{i}","{k}","dram__bytes_write.sum","byte","0"')
        rows.append(f'"{i}","{k}","smsp__inst_executed.sum","Minst","{minst}"')
    p = tmp_path / "l.csv"
    p.write_text("==PROF== x\n" + head + "\n".join(rows) + "\n")
    s = nt.summarize(nt.read_launches(str(p)))
    assert s[8]["calls"] == 1 and s[8]["launches"] == 2
    assert abs(s[8]["dram_bytes_per_launch"] - 110e6) < 1 and abs(s[8]["us_per_launch"] - 3.0) < 1e-9
    assert abs(s[9]["warp_instructions_per_launch"] - 22e6) < 1                 # both passes: one call
    assert s[0]["launches"] == 2 and abs(s[0]["dram_bytes_per_launch"] - 10e6) < 1   # mean per launch
    assert abs(s[0]["warp_instructions_per_launch"] - 4e6) < 1


def test_ncu_scale_spec_by_number_or_name():
    from paper_0904_3662_gb300 import ncu_traffic as nt
    assert nt.parse_scale("8:18.715,10:18.715") == {8: 18.715, 10: 18.715}
    assert nt.parse_scale("grid_gather_sort:2, grid_finish:0.5") == {8: 2.0, 10: 0.5}
    assert nt.parse_scale("") == {}
    with pytest.raises(ValueError):
        nt.parse_scale("no_such_phase:2")


def test_sms_a_class_can_occupy():
    cls = np.array([0] * 20 + [2] * 3 + [7] + [5] * 50 + [8] * 2)
    used = bench.sms_used_by_class(cls, 152)
    assert used[0] == 3                  # 20 warp-class haloes, 8 per CTA
    assert used[2] == 3                  # one CTA per halo
    assert used[7] == 16                 # one 16-CTA cluster
    assert used[5] == 152                # 50 four-CTA clusters fill the GPU
    assert used[8] == 152 and 1 not in used
    e = {"warp_instructions_per_launch": 16 * 4 * 2070e6 * 1e-3 * 0.5}
    r = bench.issue_roofline(e, 1.0, 2070.0, 152, 16)
    assert abs(r["frac_of_sms_used"] - 0.5) < 1e-12 and abs(r["frac"] - 0.5 * 16 / 152) < 1e-12

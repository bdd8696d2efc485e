"""Per-phase DRAM bytes and warp instructions from an ncu launch list.

bench.py reports, beside the HBM roofline of its dominant phase, the DRAM
bytes that phase moved and the warp instructions it issued, both per launch
and both from an ncu capture of the same workload.  This module turns the CSV
that ncu writes (`--csv --log-file`) into the table bench.py reads
(profiles/traffic.json): one entry per (workload, phase), keyed to a hash of
the phase's kernel sources, so that a number taken on older kernels is not
reported for newer ones.

The capture (on the GPU machine, after the same command exited 0 without ncu):

    ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,smsp__inst_executed.sum \\
        --clock-control none --csv --log-file launches.csv \\
        python bench.py --steps 2 --warmup 3 --no-plain --no-e2e --no-cpu-baseline --no-graphs --no-tune

and then, anywhere:

    python -m paper_0904_3662_gb300.ncu_traffic launches.csv --workload batch

Phases: each on-chip size class is one kernel launch per call (the figure is
the mean over its launches); each multi-CTA phase is several kernels per call
(prepare + radix passes; the passes of the iteration; the final pass, virial
search, records and profile rows), whose figure is their sum per call, the
calls counted by the one g_scales launch each call makes (a list that a launch
count cut off inside a call is read up to its last complete call).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
from collections import defaultdict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_CSRC = "paper_0904_3662_gb300/csrc/"
_DEV = _CSRC + "ahf_device.cuh"
_ONCHIP = [_CSRC + "ahf_onchip.cu", _DEV]
_GRID = [_CSRC + "ahf_grid.cu", _DEV]
PHASE_SOURCES = {0: [_CSRC + "ahf_warp.cu", _DEV], 1: _ONCHIP, 2: _ONCHIP, 3: _ONCHIP, 4: _ONCHIP, 5: _ONCHIP,
                 6: _ONCHIP, 7: _ONCHIP, 8: _GRID, 9: _GRID, 10: _GRID, 11: [_CSRC + "ahf_profile.cu", _DEV]}
PHASE_NAMES = ("warp_512", "cta_1k", "cta_4k", "cta_8k", "cluster2_16k", "cluster4_32k", "cluster8_64k",
               "cluster16_128k", "grid_gather_sort", "grid_iterate", "grid_finish", "profile")
GRID_PHASES = (8, 9, 10)

# unbind_kernel<threads, capacity, coordinate type, cluster size> -> size class
_ONCHIP_CLASS = {(128, 1024, 1): 1, (256, 4096, 1): 2, (512, 8192, 1): 3, (512, 8192, 2): 4,
                 (512, 8192, 4): 5, (512, 8192, 8): 6, (512, 8192, 16): 7}
_GRID_KERNELS = [
    (8, r"g_prepare_|g_scales|g_hist|g_digit_scan|g_digit_base|g_scatter|g_fill_identity|g_sums|g_halo<[^,]+, (true|1),"),
    (9, r"g_pass|g_removed|g_halo<[^,]+, (false|0),"),
    (10, r"g_final|g_virial|g_result|g_rows_"),
]
# values in bytes, nanoseconds and instructions whatever unit a row names
_UNIT = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9,
         "ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
         "inst": 1.0, "Kinst": 1e3, "Minst": 1e6, "Ginst": 1e9}
METRICS = ("gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum")


def source_hash(files, root: str = ROOT) -> str:
    """First 16 hex digits of the sha256 of the files' bytes, in order."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def phase_of(kernel: str):
    """The phase a kernel belongs to, or None (the bench's L2 flush, other
    calls' kernels)."""
    if "warp_kernel" in kernel:
        return 0
    m = re.search(r"unbind_kernel<(\d+), (\d+), (\d+), (\d+)>", kernel)
    if m:
        nt, cap, _ct, cs = (int(x) for x in m.groups())
        return _ONCHIP_CLASS.get((nt, cap, cs))
    for ph, pat in _GRID_KERNELS:
        if re.search(pat, kernel):
            return ph
    if "prof_chunk" in kernel or "prof_final" in kernel:
        return 11
    return None


def read_launches(path: str):
    """[(launch id, kernel name, {metric: value})] from an ncu --csv log."""
    with open(path, newline="") as f:
        rows = list(csv.reader(f))
    head = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    h = rows[head]
    ii, ki, mi, vi = h.index("ID"), h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value")
    ui = h.index("Metric Unit") if "Metric Unit" in h else None
    per = {}
    for r in rows[head + 1:]:
        if len(r) <= vi:
            continue
        key = int(r[ii])
        e = per.setdefault(key, (r[ki], {}))
        scale = _UNIT.get(r[ui], 1.0) if ui is not None else 1.0
        e[1][r[mi]] = float(r[vi].replace(",", "")) * scale
    return [(k, v[0], v[1]) for k, v in sorted(per.items())]


def summarize(launches):
    """{phase: {kernel, launches, calls, dram_bytes_per_launch,
    warp_instructions_per_launch, us_per_launch}}; per launch = per kernel
    launch for on-chip classes, per call for the multi-CTA phases."""
    tot = defaultdict(lambda: {"n": 0, "us": 0.0, "dram": 0.0, "inst": 0.0, "have_inst": True, "names": set()})
    # a list cut off by the capture's launch count ends inside a call of the
    # multi-CTA class: keep the complete calls (each ends with one g_result)
    ends = [i for i, (_, name, _) in enumerate(launches) if "g_result" in name]
    if ends:
        last = ends[-1]
        while last + 1 < len(launches) and phase_of(launches[last + 1][1]) == 10:
            last += 1                      # the profile rows after the record
        launches = launches[:last + 1]
    calls = 0
    for _, name, m in launches:
        if "g_scales" in name:
            calls += 1
        ph = phase_of(name)
        if ph is None:
            continue
        t = tot[ph]
        t["n"] += 1
        t["us"] += m.get("gpu__time_duration.sum", 0.0) / 1e3     # ns -> us
        t["dram"] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        if "smsp__inst_executed.sum" in m:
            t["inst"] += m["smsp__inst_executed.sum"]
        else:
            t["have_inst"] = False
        t["names"].add(re.sub(r"\(.*", "", name).strip())
    out = {}
    for ph, t in sorted(tot.items()):
        per = max(calls, 1) if ph in GRID_PHASES else t["n"]
        out[ph] = {"kernel": PHASE_NAMES[ph], "launches": t["n"], "calls": per,
                   "dram_bytes_per_launch": t["dram"] / per,
                   "warp_instructions_per_launch": t["inst"] / per if t["have_inst"] else None,
                   "us_per_launch": t["us"] / per}
    return out


def parse_scale(spec: str):
    """{phase: factor} from "phase:factor,...", each phase given by its
    number or its name (e.g. "8:18.7,grid_finish:18.7")."""
    out = {}
    for kv in filter(None, (x.strip() for x in spec.split(","))):
        k, v = kv.rsplit(":", 1)
        ph = int(k) if k.strip().lstrip("-").isdigit() else PHASE_NAMES.index(k.strip())
        out[ph] = float(v)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--workload", required=True)
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "traffic.json"))
    ap.add_argument("--command", default="")
    ap.add_argument("--scale", default="",
                    help="phase:factor,... (phase number or name): entries for a workload too large to capture "
                         "under several ncu passes, scaled from a smaller case of the same kernels by the units "
                         "each phase processes")
    args = ap.parse_args()
    launches = read_launches(args.csv)
    s = summarize(launches)
    if args.scale:
        factors = parse_scale(args.scale)
        s = {ph: e for ph, e in s.items() if ph in factors}
        for ph, e in s.items():
            f = factors[ph]
            e["dram_bytes_per_launch"] *= f
            if e["warp_instructions_per_launch"] is not None:
                e["warp_instructions_per_launch"] *= f
            e["us_per_launch"] *= f
            e["scaled_from"] = f"{os.path.basename(args.csv)} x {f:g} (units processed)"
    t = {}
    if os.path.exists(args.out):
        with open(args.out) as f:
            t = json.load(f)
    if args.command:
        t["command"] = args.command
    t["note"] = ("DRAM bytes (read + write) and warp instructions per launch of each phase (per call for the "
                 "multi-CTA phases), from an ncu launch list that serialises launches with caches flushed; "
                 "bench.py reports the entry of its dominant phase while the kernel sources hash to source_hash")
    for ph, e in s.items():
        e["source_hash"] = source_hash(PHASE_SOURCES[ph])
        t[f"{args.workload}:{ph}"] = e
        inst = e["warp_instructions_per_launch"]
        print(f"{args.workload}:{ph:2d} {e['kernel']:18s} launches {e['launches']:4d} calls {e['calls']:3d} "
              f"{e['us_per_launch']:9.1f} us  {e['dram_bytes_per_launch'] / 1e6:9.2f} MB  "
              f"{(inst or 0) / 1e6:8.2f} M warp-instr")
    with open(args.out, "w") as f:
        json.dump(t, f, indent=1)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the batched unbinding stage (libahfgpu) on GB300.

One step = one pass of the whole stage over one synthetic batch: gather +
recentre + radial sort + iterated potential / escape test / removal +
virial radius and the log-radial profile, in one ahf_unbind_profile_batch
call.  Metric: particle-iterations per second, where a
particle-iteration is one member tested in one unbinding iteration (the
count every implementation of the method performs; the library reports it
per halo).

Default workload: 2,000 NFW haloes, N_p ~ N^-1.9 on [100, 1e5] plus 15 %
contaminants, float32 positions relative to each centre (about 1.8e6
particles).  Inputs (~45 MB) are smaller than L2, so a 256 MiB buffer is
written between timed steps to flush it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun each rank runs its own batch (seed +
rank): haloes are independent, there is no collective on the data path,
and the scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0904_3662_gb300 import ncu_traffic  # noqa: E402

METRIC = "particle-iterations/s"
N_BINS = 32
R_MIN_FRAC = 0.01
FLUSH_BYTES = 256 << 20


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ahf", "reference"], default="ahf")
    ap.add_argument("--workload", choices=["batch", "single", "tail", "tail4", "sweep", "serve", "latency"],
                    default="batch")
    ap.add_argument("--requests", type=int, default=50_000, help="serve workload: requests per rate")
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000",
                    help="serve workload: Poisson arrival rates (requests/s)")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain one-halo-per-launch path")
    ap.add_argument("--no-tune", action="store_true", help="library default routing (no autotuner file)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--properties", action="store_true",
                    help="also time ahf_halo_properties and ahf_match_catalogs on the step's outputs")
    ap.add_argument("--trace", action="store_true",
                    help="after timing, one traced step: per-halo phase times of the on-chip kernels")
    ap.add_argument("--no-graphs", dest="graphs", action="store_false",
                    help="plain launches instead of CUDA graph replay in the timed steps")
    return ap.parse_args()


def make_workload(name, rank):
    from paper_0904_3662_gb300 import synth
    if name == "batch":
        pop = synth.halo_batch(seed=synth.SEED_BASE + 2 + 1000 * rank)
        desc = "2000 NFW haloes, N_p ~ N^-1.9 on [1e2, 1e5] + 15% contaminants, float32 relative SoA"
    elif name == "single":
        pop = synth.single_halo(seed=synth.SEED_BASE + 1 + 1000 * rank)
        desc = "one NFW halo (1e4 particles, c=10, M=1e12) + 1e3 background, float64"
    elif name == "tail":
        pop = synth.large_tail(seed=synth.SEED_BASE + 3 + 1000 * rank)
        desc = "64 hosts of 1e6-1e7 particles + 20 subhaloes each, float32 box coordinates, 500 Mpc/h box"
    elif name == "tail4":
        pop = synth.large_tail(seed=synth.SEED_BASE + 301 + 1000 * rank, counts=[4_000_000, 3_000_000, 2_500_000,
                                                                                1_500_000])
        desc = "4 large-tail hosts of 4e6, 3e6, 2.5e6, 1.5e6 particles + 20 subhaloes each (profiling case)"
    else:
        pop = synth.precision_sweep(seed=synth.SEED_BASE + 4 + 1000 * rank)
        desc = "1e5 NFW haloes, N_p ~ N^-1.9 on [1e2, 1e5] + 10% background, float64"
    return pop, desc


# ---- distributed plumbing (barrier + max over ranks only) -------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---- clocks ------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def count(self):
        return len(self.lines)

    def wait_samples(self, n, timeout=3.0):
        """Block until the sampler has produced n lines (or the timeout)."""
        t0 = time.perf_counter()
        while self.proc and len(self.lines) < n and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---- algorithmic bytes per phase: what each phase must move at least (inputs read once,
# ---- outputs written once, the multi-CTA radial stream read once per pass) ------------

def traced_classes(ctx, step, pop):
    """The size class each halo ran in (the library may promote the haloes
    of a small batch): the class recorded by a traced step for on-chip
    haloes, the multi-CTA class for the others."""
    import torch
    from paper_0904_3662_gb300 import ahf
    ctx.set_option(ahf.OPT_TRACE, 1)
    step()
    torch.cuda.synchronize()
    ctx.sync()
    ctx.set_option(ahf.OPT_TRACE, 0)
    t = ctx.trace(pop.n_halos)
    return np.where(t[:, 0] > 0, t[:, 7] & 255, len(ahf.VARIANT_CAPS))


def es_grid(pop):
    """Bytes of a real in the multi-CTA class's streams (float in the mixed mode
    the bench runs)."""
    return 4


def phase_bytes(pop, res, cls):
    """Algorithmic HBM bytes of each phase for one step."""
    es = 8 if pop.coord_type == 0 else 4
    in_b = 6 * es + (es if pop.m is not None else 0)
    cand = pop.count.astype(np.float64)
    nb = res["n_bound"].astype(np.float64)
    nm = res["n_member"].astype(np.float64)
    pit = res["part_iter"].astype(np.float64)
    from paper_0904_3662_gb300 import ahf
    nv = len(ahf.VARIANT_CAPS)
    out = np.zeros(nv + 4)
    for v in range(nv):
        s = cls == v
        # read the candidates once, write bound list + phi + the record
        out[v] = in_b * cand[s].sum() + 12.0 * nb[s].sum() + 88.0 * s.sum()
    g = cls == nv
    # multi-CTA class: the radial-order stream holds (w, r) per member, w the
    # velocity plus the Hubble flow (4 reals), and the mass when masses differ
    stream = 4 * es_grid(pop) + (es_grid(pop) if pop.m is not None else 0)
    out[nv] = in_b * cand[g].sum() + stream * nm[g].sum()          # inputs in once, radial stream out once
    out[nv + 1] = stream * pit[g].sum()                             # the stream read once per particle-iteration
    # the stream read once more; bound list, phi, record, profile rows out
    out[nv + 2] = (stream * nm[g].sum() + (8.0 + es_grid(pop)) * nb[g].sum() + 88.0 * g.sum()
                   + 32.0 * N_BINS * g.sum())
    pos_b = 3 * es + (es if pop.m is not None else 0)
    out[nv + 3] = (pos_b + 8.0) * nb.sum() + 32.0 * N_BINS * len(nb)  # gather bound particles, write rows
    return out


def source_hash(files):
    return ncu_traffic.source_hash(files, ROOT)


PHASE_SOURCES = ncu_traffic.PHASE_SOURCES


def measured_entry(phase, workload):
    """The committed ncu figures of a phase (profiles/traffic.json), or None
    when there are none or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    e = t.get(f"{workload}:{phase}")
    if not e or e.get("source_hash") != source_hash(PHASE_SOURCES[phase]):
        return None
    return e


def measured_traffic(phase, workload):
    """DRAM bytes per launch of a phase from the committed ncu summary, or
    None when there is none or the kernel source changed since."""
    e = measured_entry(phase, workload)
    return e.get("dram_bytes_per_launch") if e else None


def issue_roofline(entry, ms_per_launch, sm_mhz, n_sm, sms_used=None):
    """Issue-slot roofline of a phase: its warp instructions (ncu) per launch
    over its live duration, against every SM sub-partition issuing one warp
    instruction per clock (SMs x 4 x SM clock).  With sms_used (the SMs the
    launch can occupy, e.g. 16 for one 16-CTA cluster) also the fraction of
    those SMs' slots.  None without a count."""
    if not entry or not entry.get("warp_instructions_per_launch") or ms_per_launch <= 0:
        return None
    inst = float(entry["warp_instructions_per_launch"])
    achieved = inst / (ms_per_launch / 1e3) / 1e9
    peak = n_sm * 4 * sm_mhz * 1e6 / 1e9
    out = {"warp_instructions": inst, "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
           "frac": achieved / peak, "peak_from": f"{n_sm} SMs x 4 issue slots x {sm_mhz:.0f} MHz"}
    if sms_used:
        out["sms_used"] = int(sms_used)
        out["frac_of_sms_used"] = achieved / (sms_used * 4 * sm_mhz * 1e6 / 1e9)
    return out


def sms_used_by_class(cls, n_sm):
    """SMs each phase's launch can occupy: an on-chip class takes one CTA
    (or one cluster of 2..16 CTAs, one per SM) per halo at most; the warp
    class packs several haloes per CTA; the multi-CTA phases span the GPU."""
    from paper_0904_3662_gb300 import ahf
    nv = len(ahf.VARIANT_CAPS)
    out = {}
    for v in range(nv):
        n = int(np.sum(cls == v))
        if n == 0:
            continue
        cs = 1 << (v - 3) if v >= 4 else 1
        per = 8 if v == 0 else 1
        out[v] = min(n_sm, ((n + per - 1) // per) * cs)
    for ph in range(nv, nv + 4):
        out[ph] = n_sm
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---- the CPU oracle as a baseline -----------------------------------------------------

def cpu_baseline(pop, sample_desc=None, budget_s=30.0):
    from oracle import ahf_oracle as O
    from paper_0904_3662_gb300 import ahf
    prm = ahf.params_for(pop)
    op = O.Params(G=prm.G, H=prm.H, delta_rho=prm.delta_rho, r_soft=prm.r_soft, box=prm.box,
                  max_iter=prm.max_iter, band=prm.band)
    # a bounded sample: haloes in input order until the budget is spent
    t0 = time.perf_counter()
    units = 0
    done = 0
    for h in range(pop.n_halos):
        r = O.unbind_population(pop, op, halos=[h], n_bins=N_BINS, r_min_frac=R_MIN_FRAC)[h]
        units += r["part_iter"]
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": sample_desc or f"first {done} of {pop.n_halos} haloes of the same workload "
                                     f"({units} particle-iterations, unbinding + profile), one process"}


def cpu_baseline_parallel(pop, n_halos, workers=None):
    """The oracle over the first n_halos haloes spread over one spawned
    process per host core; the rate uses the longest worker's compute time
    (process start-up excluded)."""
    from oracle import ahf_oracle as O
    from paper_0904_3662_gb300 import ahf
    workers = workers or os.cpu_count() or 1
    prm = ahf.params_for(pop)
    op = O.Params(G=prm.G, H=prm.H, delta_rho=prm.delta_rho, r_soft=prm.r_soft, box=prm.box,
                  max_iter=prm.max_iter, band=prm.band)
    # haloes dealt to the workers by greedy LPT on their candidate counts
    from paper_0904_3662_gb300 import shard
    chunks = [[int(h) for h in c] for c in shard.lpt_partition(pop.count[:n_halos], workers)]
    res, dt = O.unbind_population_parallel(pop, op, range(n_halos), workers, n_bins=N_BINS, r_min_frac=R_MIN_FRAC,
                                           chunks=chunks)
    units = sum(v[1] for v in res.values())
    return {"value": units / dt, "unit": METRIC, "cores": workers, "kind": "oracle",
            "sample": f"first {n_halos} of {pop.n_halos} haloes of the same workload ({units} particle-iterations, "
                      f"unbinding + profile), one process per core (LPT), longest worker's compute time"}


def run_reference(args):
    world, rank, _ = dist_init()
    if rank != 0:
        barrier(world)
        return 0
    pop, desc = make_workload(args.workload, 0)
    cb = []
    # each step: the oracle over a bounded sample of the workload
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        cpu_baseline(pop, budget_s=budget)
    vals = [cpu_baseline(pop, budget_s=budget) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "halos": pop.n_halos, "particles": pop.n_particles},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    barrier(world)
    return 0


# ---- the GPU arm -----------------------------------------------------------------------

def run_ahf(args):
    import torch
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_0904_3662_gb300 import ahf, build_lib
    build_lib.build()
    t0 = time.perf_counter()
    pop, desc = make_workload(args.workload, rank)
    log(f"workload {pop.n_halos} haloes / {pop.n_particles} particles in {time.perf_counter() - t0:.1f} s")
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    n_slots = pop.n_particles
    prof = torch.empty((pop.n_halos, N_BINS, 4), dtype=torch.float64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tuning = ensure_tuning(args, ahf, torch, local, pop, parts, hal, prm, flush)
    ctx = ahf.Context(local)
    out = ctx.alloc_outputs(pop.n_halos, n_slots, with_phi=True, with_removed=False)
    ctx.set_option(ahf.OPT_TIMING, 1)

    def step():
        ctx.unbind_profile_batch(parts, hal, prm, n_bins=N_BINS, r_min_frac=R_MIN_FRAC, out=out, prof=prof,
                                 stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.sync()
    res = ahf.results_to_numpy(out["res"])
    units = float(res["part_iter"].sum())
    cls = traced_classes(ctx, step, pop)
    pbytes = phase_bytes(pop, res, cls)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phase_ms = np.zeros(ahf.N_PHASES)
    phase_n = np.zeros(ahf.N_PHASES)
    launches = 0
    barrier(world)
    torch.cuda.synchronize()
    # steps back to back, as a caller streaming batches runs them: the host
    # prepares step i + 1 while the device runs step i; the phase events stay
    # off here (reading them needs a host wait per step).  The batch repeats,
    # so its launches run as a CUDA graph (captured in an untimed step)
    ctx.set_option(ahf.OPT_TIMING, 0)
    ctx.set_option(ahf.OPT_GRAPHS, 1 if args.graphs else 0)
    for _ in range(2):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.wait_samples(1)                       # the sampler is up before the timed steps
        n0 = clk.count()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()                         # L2 flush, outside the timed events
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        # a timed region shorter than the sampling period gets no sample of
        # its own: the same steps keep the GPU under the same load (untimed)
        # until two samples fall after the start of the timed steps
        t_hold = time.perf_counter()
        while clk.count() < n0 + 2 and time.perf_counter() - t_hold < 3.0:
            for _ in range(20):
                flush.zero_()
                step()
            torch.cuda.synchronize()
        clk.lines = clk.lines[n0:]
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # the same steps again with per-phase events (one host wait per step) for
    # the per-kernel durations the roofline uses: the classes one after
    # another, each kernel timed alone as in the ncu launch list
    ctx.set_option(ahf.OPT_GRAPHS, 0)
    ctx.set_option(ahf.OPT_TIMING, 1)
    ctx.set_option(ahf.OPT_SERIAL, 1)
    for i in range(args.steps):
        flush.zero_()
        step()
        st = ctx.stats()
        launches += st["launches"]
        for k in range(ahf.N_PHASES):
            if st["phase_ms"][k] >= 0:
                phase_ms[k] += st["phase_ms"][k]
                phase_n[k] += 1
    ctx.set_option(ahf.OPT_SERIAL, 0)
    ms = float(np.mean(step_ms))
    ms_max = reduce_max(world, ms)
    total_units = reduce_sum(world, units)
    value = total_units / (ms_max / 1e3)

    # roofline of the dominant phase (device time per launch of that phase)
    avg = np.where(phase_n > 0, phase_ms / np.maximum(phase_n, 1), 0.0)
    dom = int(np.argmax(avg))
    peak, peak_kind = peaks()
    achieved = pbytes[dom] / (avg[dom] / 1e3) / 1e9 if avg[dom] > 0 else 0.0
    entry = measured_entry(dom, args.workload)
    traffic = entry.get("dram_bytes_per_launch") if entry else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": ahf.PHASE_NAMES[dom], "algorithmic_bytes": float(pbytes[dom]),
                "ms_per_launch": float(avg[dom]), "peak_source": peak_kind,
                "durations": "each size class timed alone (AHF_OPT_SERIAL), L2 flushed before the step",
                "phases_ms": {ahf.PHASE_NAMES[k]: round(float(avg[k]), 4) for k in range(ahf.N_PHASES)
                              if phase_n[k] > 0}}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
            "config": {"workload": desc, "halos": pop.n_halos, "particles": pop.n_particles,
                       "particle_iterations_per_step": units, "l2": "flushed (256 MiB write) between steps",
                       "parallelism": f"replicas x{world}, haloes independent, no collective",
                       "launch": "CUDA graph replay (AHF_OPT_GRAPHS)" if args.graphs else "plain launches"},
            "gpu_launches": launches, "roofline": roofline,
            "timed_wall_s": t_wall, "tuning": tuning}
    clocks = clk.summary()
    if clocks:
        clocks["window"] = "the timed steps and the same steps right after them (200 ms sampling)"
    line["clocks"] = clocks
    # the same phase against the issue slots (on-chip classes are issue- and
    # latency-bound rather than HBM-bound), and every phase with a count
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = float(clocks["sm_mhz"]) if clocks else 2070.0
    used = sms_used_by_class(cls, n_sm)
    roofline["issue"] = issue_roofline(entry, float(avg[dom]), sm_mhz, n_sm, used.get(dom))
    roofline["issue_by_phase"] = {
        ahf.PHASE_NAMES[k]: {"frac": round(r["frac"], 4), "sms_used": r.get("sms_used"),
                             "frac_of_sms_used": round(r.get("frac_of_sms_used", r["frac"]), 4)}
        for k in range(ahf.N_PHASES) if phase_n[k] > 0
        for r in [issue_roofline(measured_entry(k, args.workload), float(avg[k]), sm_mhz, n_sm, used.get(k))] if r}
    if rank == 0 and args.properties:
        line["properties"] = time_properties(ctx, parts, hal, prm, pop, stream, flush)
        log(f"properties {line['properties']['properties_ms']:.3f} ms, matching {line['properties']['match_ms']:.3f} ms")
    if args.trace:
        from paper_0904_3662_gb300 import trace_report
        ctx.set_option(ahf.OPT_TIMING, 0)
        ctx.set_option(ahf.OPT_TRACE, 1)
        flush.zero_()
        step()
        summary = trace_report.summarize(ctx.trace(pop.n_halos))
        ctx.set_option(ahf.OPT_TRACE, 0)
        line["trace"] = summary
        log("trace (us):\n" + trace_report.table(summary))

    log(f"timed {args.steps} steps: {ms:.3f} ms/step, {value:.4g} {METRIC}")
    if rank == 0 and not args.no_plain:
        line["plain"] = time_plain(ctx, parts, hal, prm, out, stream, units, flush)
        line["plain"]["batched_speedup"] = (units / (ms / 1e3)) / line["plain"]["value"]
        log(f"plain path {line['plain']['ms_per_step']:.1f} ms/step")
    if rank == 0 and not args.no_e2e:
        line["e2e"] = time_e2e(ctx, pop, hal, prm, units, args)
        log(f"e2e {line['e2e']['ms_per_step']:.2f} ms/step")
    if rank == 0 and not args.no_cpu_baseline:
        one = cpu_baseline(pop)
        n_done = int(one["sample"].split()[1])
        line["cpu_baseline"] = cpu_baseline_parallel(pop, n_done)
        line["cpu_baseline"]["one_core"] = {"value": one["value"], "sample": one["sample"]}
        log(f"cpu baseline {line['cpu_baseline']['value']:.4g} {METRIC} on {line['cpu_baseline']['cores']} cores, "
            f"{one['value']:.4g} on one")
    if rank == 0:
        print(json.dumps(line))
    barrier(world)
    return 0


def ensure_tuning(args, ahf, torch, local, pop, parts, hal, prm, flush):
    """The routing the step runs with: the autotuner's file for this device
    and build (paper_0904_3662_gb300/tuning/<device>.txt), made first by a
    bounded search on this workload when it is missing or stale (the default
    batch workload only), and handed to the library through AHF_TUNING."""
    from paper_0904_3662_gb300 import autotune
    if args.no_tune:
        os.environ.pop("AHF_TUNING", None)
        return {"file": None, "options": "library defaults"}
    key = autotune.device_key(torch.cuda.get_device_name(local))
    path = autotune.tuning_path(key)
    build = ahf.build_id()
    made = False
    if not autotune.valid_for(path, key, build) and args.workload == "batch":
        ctx = ahf.Context(local)
        ctx.set_option(ahf.OPT_GRAPHS, 1)
        out = ctx.alloc_outputs(pop.n_halos, pop.n_particles, with_phi=True, with_removed=False)
        prof = torch.empty((pop.n_halos, N_BINS, 4), dtype=torch.float64, device="cuda")

        def step():
            ctx.unbind_profile_batch(parts, hal, prm, n_bins=N_BINS, r_min_frac=R_MIN_FRAC, out=out, prof=prof)

        t0 = time.perf_counter()
        cfg, d, t, trials = autotune.tune(ctx, step, ahf, bool(pop.count.max() > ahf.VARIANT_CAPS[-1]), flush,
                                          budget_s=45.0, log=log)
        autotune.write(path, key, build, cfg, f"2,000-halo batch; default {d:.4f} ms, tuned {t:.4f} ms, "
                                              f"{len(trials)} settings timed")
        log(f"autotune: default {d:.4f} ms, tuned {t:.4f} ms ({len(trials)} settings, "
            f"{time.perf_counter() - t0:.0f} s)")
        made = True
        del ctx
    if not autotune.valid_for(path, key, build):
        os.environ.pop("AHF_TUNING", None)
        return {"file": None, "options": "library defaults (no tuning for this device and build)"}
    os.environ["AHF_TUNING"] = path
    t = autotune.read(path)
    names = {ahf.OPT_PROMOTE: "promote", ahf.OPT_PASS_CHUNK: "pass_chunk"}
    names.update({ahf.OPT_CLASS_CUT + v: f"class_cut_{ahf.PHASE_NAMES[v]}" for v in range(len(ahf.VARIANT_CAPS))})
    return {"file": os.path.relpath(path, ROOT), "build": build, "made_in_this_run": made,
            "options": {names.get(o, str(o)): v for o, v in t["options"].items()}, "note": t["comment"]}


def time_properties(ctx, parts, hal, prm, pop, stream, flush, steps=5):
    """ahf_halo_properties over the step's outputs, and ahf_match_catalogs of
    the catalogue with itself (device time per call, after a warm-up)."""
    import torch
    from paper_0904_3662_gb300 import ahf
    out = ctx.unbind_batch(parts, hal, prm, stream=stream)
    torch.cuda.synchronize()
    res = ahf.results_to_numpy(out["res"])
    off = torch.from_numpy(pop.offset.astype(np.int64)).cuda()
    cnt = torch.from_numpy(res["n_bound"].astype(np.int64)).cuda()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))
    t_p = timed(lambda: ctx.halo_properties(parts, hal, prm, out, stream=stream))
    t_m = timed(lambda: ctx.match_catalogs(pop.n_particles, out["bound_idx"], off, cnt, out["bound_idx"], off, cnt,
                                           stream=stream))
    return {"properties_ms": t_p, "match_ms": t_m,
            "what": "ahf_halo_properties on the batch's bound sets; ahf_match_catalogs of the catalogue with itself"}


def time_plain(ctx, parts, hal, prm, out, stream, units, flush, steps=2):
    """The plain one-halo-per-launch form on the same inputs (fewer steps: it
    is slow by design)."""
    import torch
    ctx.unbind_batch(parts, hal, prm, out=out, stream=stream, plain=True)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.unbind_batch(parts, hal, prm, out=out, stream=stream, plain=True)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    return {"value": units / (ms / 1e3), "unit": METRIC, "ms_per_step": ms, "steps": steps,
            "what": "ahf_unbind_plain: one halo at a time, separate launches per step, host sync per iteration "
                    "(unbinding only, no profile)"}


def time_e2e(ctx, pop, hal, prm, units, args):
    """The same step through ahf_unbind_batch_host: pinned host inputs in,
    results back in host memory, copies inside the timed region."""
    import torch
    from paper_0904_3662_gb300 import ahf

    def pinned(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a)
        t = torch.from_numpy(a.reshape(-1).view(np.uint8)).pin_memory()
        return t.numpy().view(a.dtype).reshape(a.shape)
    hp = ahf.Particles(pinned(pop.x), pinned(pop.y), pinned(pop.z), pinned(pop.vx), pinned(pop.vy),
                       pinned(pop.vz), pinned(pop.m), pop.m0, pop.coord_type)
    n = pop.n_particles
    out = {"res": pinned(np.zeros(pop.n_halos, dtype=ahf.RESULT_DTYPE)),
           "bound_idx": pinned(np.zeros(n, dtype=np.int64)), "phi": pinned(np.zeros(n, dtype=np.float32)),
           "removed_iter": None, "prof": pinned(np.zeros((pop.n_halos, N_BINS, 4)))}
    es = hp.x.dtype.itemsize
    h2d = 6 * n * es + (n * es if pop.m is not None else 0) + hal.nbytes
    d2h = out["res"].nbytes + out["bound_idx"].nbytes + out["phi"].nbytes + out["prof"].nbytes
    def timed():
        for _ in range(max(1, args.warmup)):
            ctx.unbind_batch_host(hp, hal, prm, out=out, n_bins=N_BINS, r_min_frac=R_MIN_FRAC)
        ts = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            ctx.unbind_batch_host(hp, hal, prm, out=out, n_bins=N_BINS, r_min_frac=R_MIN_FRAC)
            ts.append(time.perf_counter() - t0)
        return float(np.mean(ts))
    # the library's default route for page-locked buffers, then the others
    # for comparison (0: staged copies, 1: in place, 2: per-class pulls)
    default = ctx.get_option(ahf.OPT_HOST_DIRECT)
    modes = {}
    for mode in (default, *(m for m in (0, 1, 2) if m != default)):
        ctx.set_option(ahf.OPT_HOST_DIRECT, mode)
        modes[mode] = timed()
    ctx.set_option(ahf.OPT_HOST_DIRECT, default)
    s = modes[default]
    names = {0: "staged copies", 1: "buffers used in place",
             2: "inputs read in place, outputs pushed per size class"}
    return {"value": units / s, "unit": METRIC, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": s * 1e3,
            "ms_per_step_by_route": {names[m]: round(v * 1e3, 4) for m, v in sorted(modes.items())},
            "api": f"ahf_unbind_batch_host (unbinding + profile, page-locked host buffers, {names[default]})"}


def run_serve(args):
    """Serving stream: Poisson arrivals of one-halo requests (95 % with
    N_p ~ N^-1.9 on [100, 1e4), 5 % on [1e4, 1e5], 15 % contaminants each)
    submitted from host memory through ahf_serve_submit at each rate of the
    sweep; latency is the library's submit-to-poll-visible time."""
    import collections
    import torch
    from paper_0904_3662_gb300 import ahf, build_lib, synth
    build_lib.build()
    torch.cuda.init()
    t0 = time.perf_counter()
    small = synth.halo_batch(seed=synth.SEED_BASE + 5, n_halos=1900, n_lo=100, n_hi=9_999)
    large = synth.halo_batch(seed=synth.SEED_BASE + 6, n_halos=100, n_lo=10_000, n_hi=100_000)
    t_unit, counts = synth.serving_stream(n_requests=args.requests, rate_hz=1.0)
    big = counts >= 10_000
    pools = []
    for pop in (small, large):
        parts = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, pop.m0, pop.coord_type)
        hal = ahf.halos_from_population(pop)
        pools.append([ahf.Serve.request(parts, hal[h:h + 1]) for h in range(pop.n_halos)])
    reqs, reqs_src, k_small, k_big, cand = [], [], 0, 0, 0
    for b in big:
        if b:
            reqs.append(pools[1][k_big % len(pools[1])])
            reqs_src.append((large, k_big % large.n_halos))
            cand += int(large.count[k_big % large.n_halos])
            k_big += 1
        else:
            reqs.append(pools[0][k_small % len(pools[0])])
            reqs_src.append((small, k_small % small.n_halos))
            cand += int(small.count[k_small % small.n_halos])
            k_small += 1
    log(f"serve pool ready in {time.perf_counter() - t0:.1f} s; {len(reqs)} requests, {cand} candidates")
    prm = ahf.params_for(small)
    srv = ahf.Serve(prm, hbm_cap_bytes=60 << 30, coord_type=small.coord_type, m0=small.m0)
    # warm-up: a few hundred requests at no particular rate
    warm = [srv.submit_prepared(reqs[i]) for i in range(min(300, len(reqs)))]
    for rid in warm:
        while rid is not None and srv.poll(rid) is None:
            time.sleep(1e-4)
    sweep = []
    for rate in [float(r) for r in args.rates.split(",")]:
        arr = t_unit / rate
        srv.reset_stats()
        pending = collections.deque()
        refused, i, n = 0, 0, len(reqs)
        rid = 0
        start = time.perf_counter()
        with ClockSampler(torch.cuda.current_device()) as clk:
            while i < n:
                now = time.perf_counter() - start
                if now >= arr[i]:
                    rid = srv.submit_prepared(reqs[i])
                    if rid is None:
                        refused += 1
                    else:
                        pending.append(rid)
                        i += 1
                        continue
                while pending and srv.poll(pending[0]) is not None:
                    pending.popleft()
            t_sub = time.perf_counter() - start
            while pending:
                if srv.poll(pending[0]) is None:
                    time.sleep(1e-4)
                else:
                    pending.popleft()
        st = srv.stats()
        row = {"rate": rate, "offered": n / t_sub, "throughput": st["throughput"], "p50_us": st["p50_us"],
               "p99_us": st["p99_us"], "batches": st["batches"], "mean_batch": n / max(1, st["batches"]),
               "refused": refused, "clocks": clk.summary()}
        log(f"rate {rate:.0f}/s: offered {row['offered']:.0f}/s, {st['throughput']:.0f} req/s, "
            f"p50 {st['p50_us']:.0f} us, p99 {st['p99_us']:.0f} us, {st['batches']} batches")
        sweep.append(row)
    srv.close()
    plain = time_plain_requests(reqs_src, ahf, prm, sweep, t_unit)
    best = max(sweep, key=lambda r: r["throughput"])
    line = {"metric": "requests/s", "value": best["throughput"], "unit": "requests/s", "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64",
            "data": "synthetic",
            "config": {"workload": "Poisson stream of one-halo requests, 95% N_p on [100, 1e4), 5% on [1e4, 1e5], "
                                   "+15% contaminants, float32 relative, HBM cap 60 GB",
                       "requests_per_rate": len(reqs), "candidates_per_pass": cand},
            "sweep": sweep, "plain": plain}
    print(json.dumps(line))
    return 0


def time_plain_requests(reqs_src, ahf, prm, sweep, t_unit):
    """The plain launch-per-request arm on the same request stream: each
    request alone, from host memory, through the one-halo-per-launch form
    (ahf_unbind_plain: separate gather / sort / pass kernels, a host wait on
    every pass's change flag): its candidates copied in from page-locked host
    memory, the unbinding, its record and bound list copied back.  Every
    request's service time is measured on the GPU machine back to back (wall
    clock, a stream synchronisation on both sides); a single FIFO server with
    those service times then gives each request's latency (completion minus
    arrival) for the arrival times of every rate of the sweep."""
    import torch
    dev = torch.device("cuda")
    pinned = {}
    for pop, _ in reqs_src:
        if id(pop) not in pinned:
            pinned[id(pop)] = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                               for a in (pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz)]
    nmax = max(int(pop.count[h]) for pop, h in reqs_src)
    stage = [torch.empty(nmax, dtype=torch.float32, device=dev) for _ in range(6)]
    ctx = ahf.Context(0)
    out = ctx.alloc_outputs(1, nmax, with_phi=False, with_removed=False)
    res_h = torch.empty(ahf.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    bound_h = torch.empty(nmax, dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream()
    service = np.empty(len(reqs_src))
    for i, (pop, h) in enumerate(reqs_src):
        o, n = int(pop.offset[h]), int(pop.count[h])
        hal = ahf.halos_from_population(pop)[h:h + 1].copy()
        hal["offset"] = 0
        src = pinned[id(pop)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a in range(6):
            stage[a][:n].copy_(src[a][o:o + n], non_blocking=True)
        parts = ahf.Particles(*[t[:n] for t in stage], None, pop.m0, pop.coord_type)
        ctx.unbind_batch(parts, hal, prm, out=out, stream=stream, plain=True)
        res_h.copy_(out["res"], non_blocking=True)
        bound_h[:n].copy_(out["bound_idx"][:n], non_blocking=True)
        torch.cuda.synchronize()
        service[i] = time.perf_counter() - t0
    rows = []
    for r in sweep:
        arr = t_unit / r["rate"]
        done = 0.0
        lat = np.empty(len(arr))
        for i in range(len(arr)):
            done = max(arr[i], done) + service[i]
            lat[i] = done - arr[i]
        rows.append({"rate": r["rate"], "throughput": len(arr) / (done - arr[0]),
                     "p50_us": float(np.percentile(lat, 50, method="inverted_cdf") * 1e6),
                     "p99_us": float(np.percentile(lat, 99, method="inverted_cdf") * 1e6)})
        log(f"plain at {r['rate']:.0f}/s: {rows[-1]['throughput']:.0f} req/s, p50 {rows[-1]['p50_us']:.0f} us, "
            f"p99 {rows[-1]['p99_us']:.0f} us")
    return {"api": "ahf_unbind_plain per request, candidates from page-locked host memory, record and bound list "
                   "copied back", "service_us_mean": float(service.mean() * 1e6),
            "service_us_p50": float(np.median(service) * 1e6),
            "latency": "FIFO single server with the measured per-request service times, same arrival stream",
            "sweep": rows}


def run_latency(args):
    """Latency of one call for small batches, each size class as small as
    possible (AHF_OPT_PROMOTE off) and with latency promotion (on): median
    CUDA-event time of back-to-back calls with graph replay."""
    import torch
    from paper_0904_3662_gb300 import ahf, synth
    cases = [("one NFW halo, 11,000 candidates (float64)", synth.single_halo(seed=synth.SEED_BASE + 1))]
    for n_lo, n_hi, nh in ((200, 400, 1), (4000, 6000, 1), (1500, 2500, 8), (20000, 30000, 2), (100, 100_000, 20),
                           (100, 100_000, 100), (100, 100_000, 400)):
        cases.append((f"{nh} haloes, N_p on [{n_lo}, {n_hi}]", synth.halo_batch(seed=11 + nh + n_lo, n_halos=nh,
                                                                           n_lo=n_lo, n_hi=n_hi)))
    rows = []
    for desc, pop in cases:
        r = {"batch": desc, "haloes": pop.n_halos, "candidates": int(pop.count.sum())}
        for promote in (0, 1):
            ctx = ahf.Context(0)
            ctx.set_option(ahf.OPT_PROMOTE, promote)
            ctx.set_option(ahf.OPT_GRAPHS, 1)
            parts = ahf.particles_from_population(pop)
            hal = ahf.halos_from_population(pop)
            prm = ahf.params_for(pop)
            out = ctx.alloc_outputs(len(hal), pop.n_particles)
            prof = torch.empty((len(hal), N_BINS, 4), dtype=torch.float64, device="cuda")
            for _ in range(max(3, args.warmup)):
                ctx.unbind_profile_batch(parts, hal, prm, n_bins=N_BINS, r_min_frac=R_MIN_FRAC, out=out, prof=prof)
            torch.cuda.synchronize()
            ts = []
            for _ in range(args.steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                ctx.unbind_profile_batch(parts, hal, prm, n_bins=N_BINS, r_min_frac=R_MIN_FRAC, out=out, prof=prof)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b) * 1e3)
            st = ctx.stats()["phase_halos"][:len(ahf.VARIANT_CAPS)]
            key = "promoted" if promote else "smallest_class"
            r[key + "_us"] = float(np.median(ts))
            r[key + "_classes"] = {ahf.PHASE_NAMES[k]: int(n) for k, n in enumerate(st) if n}
        rows.append(r)
        log(f"{desc}: {r['smallest_class_us']:.1f} us -> {r['promoted_us']:.1f} us")
    print(json.dumps({"metric": "call latency", "unit": "us", "higher_is_better": False, "data": "synthetic",
                      "steps": args.steps, "rows": rows}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "latency":
        return run_latency(args)
    return run_ahf(args)


if __name__ == "__main__":
    sys.exit(main())

"""Autotuner of libahfgpu's routing knobs, cached per device and build.

What it tunes (every choice gives the same results bit for bit, because the
sums are exact fixed point; only the time changes):

* the size-class cut-offs: the largest candidate count each on-chip variant
  takes (AHF_OPT_CLASS_CUT + v), i.e. which shape -- one warp, one CTA of
  128 / 256 / 512 threads, a cluster of 2..16 CTAs -- a halo of a given size
  runs in, and from which size on haloes go to the multi-CTA class;
* the latency-promotion rule (AHF_OPT_PROMOTE): whether a batch that would
  leave SMs idle moves its haloes to larger classes;
* the multi-CTA class's pass chunk (AHF_OPT_PASS_CHUNK): passes enqueued
  between reads of the active count.

Search: coordinate descent from the library's defaults.  Each candidate
setting is timed on the caller's workload with CUDA events (median of `reps`
calls, each after an L2 flush); a change is kept when it is faster by more
than `min_gain`.  The result is written as a small text file keyed by the
device name and the library's build id (ahf_build_id()), which ahf_create
applies when the environment variable AHF_TUNING names it:

    device NVIDIA_GB300
    build 24721a51cc44c629
    # workload ...; default 0.331 ms, tuned 0.325 ms
    option 8 1
    option 16 512
    ...

    python -m paper_0904_3662_gb300.autotune            # tune on the 2,000-halo batch
"""
from __future__ import annotations

import os
import re
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")


def device_key(name: str) -> str:
    """The device name as ahf_create compares it: every character outside
    [A-Za-z0-9._-] replaced by '_'."""
    return re.sub(r"[^A-Za-z0-9._-]", "_", name)


def tuning_path(key: str) -> str:
    return os.path.join(TUNING_DIR, f"{key}.txt")


def write(path: str, key: str, build: str, options: dict, comment: str = "") -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(f"device {key}\nbuild {build}\n")
        for line in comment.splitlines():
            f.write(f"# {line}\n")
        for opt in sorted(options):
            f.write(f"option {int(opt)} {int(options[opt])}\n")


def read(path: str) -> dict:
    """{'device': ..., 'build': ..., 'options': {number: value}, 'comment': [...]}"""
    out = {"device": None, "build": None, "options": {}, "comment": []}
    with open(path) as f:
        for line in f:
            w = line.split()
            if not w:
                continue
            if w[0].startswith("#"):
                out["comment"].append(line[1:].strip())
            elif w[0] == "device" and len(w) == 2:
                out["device"] = w[1]
            elif w[0] == "build" and len(w) == 2:
                out["build"] = w[1]
            elif w[0] == "option" and len(w) == 3:
                out["options"][int(w[1])] = int(w[2])
            else:
                raise ValueError(f"{path}: cannot read {line!r}")
    return out


def valid_for(path: str, key: str, build: str) -> bool:
    if not os.path.exists(path):
        return False
    t = read(path)
    return t["device"] == key and t["build"] == build


def knobs(ahf, multi_cta: bool):
    """(option, candidate values) in search order; the first value of each
    list is the library's default."""
    ks = [(ahf.OPT_PROMOTE, [1, 0])]
    caps = ahf.VARIANT_CAPS
    for v in range(len(caps) - 1):
        c = caps[v]
        ks.append((ahf.OPT_CLASS_CUT + v, [c, (7 * c) // 8, (3 * c) // 4, (5 * c) // 8, c // 2]))
    if multi_cta:
        ks.append((ahf.OPT_PASS_CHUNK, [8, 4, 16]))
    return ks


def time_call(ctx, step, flush, reps: int = 15, warm: int = 3) -> float:
    """Median device time (ms) of step() over `reps` calls enqueued back to
    back (as a caller streaming batches runs them: the host prepares the
    next call while the device runs this one), each after a write of `flush`
    (an L2-sized buffer) outside the timed events, after `warm` untimed
    calls."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def tune(ctx, step, ahf, multi_cta: bool, flush, reps: int = 15, sweeps: int = 3, min_gain: float = 0.01,
         budget_s: float = 60.0, log=None):
    """Coordinate descent over knobs(); returns (options, default_ms, tuned_ms, trials)."""
    t_start = time.perf_counter()
    ks = knobs(ahf, multi_cta)
    cfg = {opt: vals[0] for opt, vals in ks}
    for opt, val in cfg.items():
        ctx.set_option(opt, val)
    best = default = time_call(ctx, step, flush, reps)
    trials = [(dict(cfg), best)]
    for _ in range(sweeps):
        improved = False
        for opt, vals in ks:
            for val in vals:
                if val == cfg[opt] or time.perf_counter() - t_start > budget_s:
                    continue
                ctx.set_option(opt, val)
                t = time_call(ctx, step, flush, reps)
                trials.append(({**cfg, opt: val}, t))
                if t < best * (1.0 - min_gain):
                    best, cfg[opt], improved = t, val, True
                    if log:
                        log(f"autotune: option {opt} = {val}: {t:.4f} ms")
                ctx.set_option(opt, cfg[opt])
        if not improved:
            break
    return cfg, default, best, trials


def main():
    import argparse
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_0904_3662_gb300 import ahf, build_lib, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--budget", type=float, default=60.0)
    args = ap.parse_args()
    build_lib.build()
    pop = synth.halo_batch(seed=synth.SEED_BASE + 2)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    out = ctx.alloc_outputs(pop.n_halos, pop.n_particles, with_phi=True, with_removed=False)
    prof = torch.empty((pop.n_halos, 32, 4), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 18, dtype=torch.float32, device="cuda")
    ctx.set_option(ahf.OPT_GRAPHS, 1)

    def step():
        ctx.unbind_profile_batch(parts, hal, prm, n_bins=32, r_min_frac=0.01, out=out, prof=prof)

    cfg, d, t, _ = tune(ctx, step, ahf, bool(pop.count.max() > ahf.VARIANT_CAPS[-1]), flush,
                        budget_s=args.budget, log=print)
    key = device_key(torch.cuda.get_device_name(0))
    path = args.out or tuning_path(key)
    write(path, key, ahf.build_id(), cfg, f"2,000-halo batch; default {d:.4f} ms, tuned {t:.4f} ms")
    print(f"{path}: default {d:.4f} ms, tuned {t:.4f} ms")


if __name__ == "__main__":
    main()

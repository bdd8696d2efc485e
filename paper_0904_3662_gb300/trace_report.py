"""Summary of a per-halo trace (ahf_get_trace, AHF_OPT_TRACE).

Each traced halo has its first thread's global-timer readings at the phase
boundaries of the on-chip kernels: start, gathered, sorted, filled,
iterated, done; the SM of that thread; and variant + 256 * iterations.
"""
from __future__ import annotations

import numpy as np

from paper_0904_3662_gb300 import ahf

PHASES = (("gather", 0, 1), ("sort", 1, 2), ("fill", 2, 3), ("iterate", 3, 4), ("emit", 4, 5))


def summarize(trace):
    """Per-variant mean / max phase durations (us), iterations, first start
    and last end relative to the earliest start, and the span of the whole
    batch."""
    t = np.asarray(trace, dtype=np.int64)
    done = t[:, 5] > 0
    if not np.any(done):
        return {"haloes": 0}
    t = t[done]
    t0 = int(t[:, 0].min())
    variant = t[:, 7] & 255
    iters = t[:, 7] >> 8
    out = {"haloes": int(t.shape[0]), "span_us": (int(t[:, 5].max()) - t0) / 1e3, "variants": {}}
    for v in np.unique(variant):
        s = t[variant == v]
        row = {"haloes": int(s.shape[0]), "iterations_mean": float(iters[variant == v].mean()),
               "first_start_us": (int(s[:, 0].min()) - t0) / 1e3, "last_end_us": (int(s[:, 5].max()) - t0) / 1e3,
               "halo_us_mean": float((s[:, 5] - s[:, 0]).mean()) / 1e3,
               "halo_us_max": float((s[:, 5] - s[:, 0]).max()) / 1e3}
        for name, a, b in PHASES:
            d = (s[:, b] - s[:, a]) / 1e3
            row[name + "_us_mean"] = float(d.mean())
        out["variants"][ahf.PHASE_NAMES[int(v)]] = row
    return out


def table(summary):
    """The summary as a markdown table."""
    cols = ["haloes", "iterations_mean"] + [n + "_us_mean" for n, _, _ in PHASES] + [
        "halo_us_mean", "halo_us_max", "first_start_us", "last_end_us"]
    lines = ["| variant | " + " | ".join(cols) + " |", "|---" * (len(cols) + 1) + "|"]
    for name, row in summary.get("variants", {}).items():
        cells = []
        for c in cols:
            v = row[c]
            cells.append(f"{v:d}" if isinstance(v, int) else f"{v:.1f}")
        lines.append(f"| {name} | " + " | ".join(cells) + " |")
    return "\n".join(lines)

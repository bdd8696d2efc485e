"""Write the oracle's summary of the single-halo workload to single_halo.json.

Calls only the seeded generator and the CPU oracle.  The stored values are a
regression record of the oracle (the oracle itself is pinned by the tests in
test_oracle_pins.py, not by this file).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ahf_oracle as O                      # noqa: E402
from paper_0904_3662_gb300 import synth                 # noqa: E402


def summary():
    pop = synth.single_halo()
    o = O.unbind_population(pop, O.Params(), n_bins=8, r_min_frac=0.01)[0]
    return {
        "workload": pop.name,
        "n_member": o["n_member"], "n_bound": int(o["order"].shape[0]),
        "n_iter": o["n_iter"], "part_iter": o["part_iter"], "status": o["status"],
        "r_vir": o["r_vir"], "m_vir": o["m_vir"], "k_vir": o["k_vir"],
        "vbulk": [float(x) for x in o["vbulk"]],
        "removed_per_iter": [int((o["removed_iter"] == t).sum()) for t in range(1, o["n_iter"] + 1)],
        "phi_first_last": [float(o["phi"][0]), float(o["phi"][-1])],
        "profile_counts": [int(c) for c in o["profile"][:, 0]],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "single_halo.json"), "w") as f:
        json.dump(summary(), f, indent=1)
        f.write("\n")

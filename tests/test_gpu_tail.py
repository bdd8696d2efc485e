"""Hosts of the large-tail workload at its own sizes: two hosts of 2.6e6 and
1.1e6 candidates (1,270 and 538 tiles of 2,048), each with its 20 subhaloes,
float32 box coordinates in the 5e5 kpc/h periodic box.  Both go through the
multi-CTA class (every tile loop, the carried chunks of the per-halo digit
and tile scans, the digit bases and scatter offsets at these sizes) in the
mixed and the all-FP64 mode, and every candidate is compared with the oracle
(Sect. 2.1 and Appendix A): removal iteration, bound set, phi, M_vir, R_vir,
v_bulk; the profile rows of the bench's call in the mixed mode."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu
from tests.parity import check_profiles, compare, fp64_rtol

pytestmark = pytest.mark.gpu

COUNTS = [2_600_000, 1_100_000]


@pytest.fixture(scope="module")
def tail_pop():
    return synth.large_tail(seed=synth.SEED_BASE + 300, counts=COUNTS)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_tail_hosts_full_size(tail_pop, mode):
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = tail_pop
    assert pop.coord_type == synth.COORD_F32_BOX and pop.box == 5e5
    prec = ahf.PREC_MIXED if mode == "mixed" else ahf.PREC_FP64
    tol = 1e-5 if mode == "mixed" else fp64_rtol(pop)
    prm = ahf.params_for(pop, precision=prec)
    out, prm, ctx, _ = run_gpu(pop, params=prm)
    st = ctx.stats()
    # both hosts ran in the multi-CTA class
    assert st["phase_halos"][ahf.PHASE_NAMES.index("grid_gather_sort")] == 2
    s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=tol,
                vir_rtol=tol, exact_order=(mode == "fp64"))
    res = out["res"]
    assert np.all(res["n_member"] >= np.asarray(COUNTS) - 10)
    assert np.all(res["n_bound"] > 0.9 * res["n_member"])
    assert s["worst_phi_rel"] <= tol
    print(f"\n{mode}: {s}")


def test_tail_hosts_profile_rows(tail_pop):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = tail_pop
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    out = ctx.unbind_profile_batch(parts, hal, prm, n_bins=32, r_min_frac=0.01)
    torch.cuda.synchronize()
    ctx.sync()
    res = ahf.results_to_numpy(out["res"])
    compare(pop, prm, res, out["bound_idx"].cpu().numpy(), out["phi"].cpu().numpy(),
            out["removed_iter"].cpu().numpy())
    check_profiles(pop, prm, res, out["prof"].cpu().numpy(), 32, 0.01)

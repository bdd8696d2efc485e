"""The 2,000-halo batch at its full size, in the launch configuration bench.py
times (ahf_unbind_profile_batch, 32 bins from 0.01 r_vir): every halo against
the oracle (removal iteration of every candidate, bound sets, phi, M_vir,
R_vir, v_bulk, profile rows), and properties that hold for every halo at any
size."""
import math

import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu
from tests.parity import check_profiles, compare

pytestmark = pytest.mark.gpu

N_BINS, R_MIN_FRAC = 32, 0.01


def _sample(counts, per_class=4, seed=7):
    """The largest halo of every size class and a few random ones."""
    caps = [0, 512, 1024, 4096, 8192, 16384, 32768, 65536, 131072, 1 << 62]
    rng = np.random.default_rng(seed)
    out = []
    for lo, hi in zip(caps[:-1], caps[1:]):
        idx = np.where((counts > lo) & (counts <= hi))[0]
        if len(idx) == 0:
            continue
        out.append(int(idx[np.argmax(counts[idx])]))
        out += [int(h) for h in rng.choice(idx, size=min(per_class, len(idx)), replace=False)]
    return sorted(set(out))


def test_full_batch_every_halo():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=synth.SEED_BASE + 2)
    assert pop.n_halos == 2000 and pop.n_particles == 1_799_222
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    out = ctx.unbind_profile_batch(parts, hal, prm, n_bins=N_BINS, r_min_frac=R_MIN_FRAC)
    torch.cuda.synchronize()
    ctx.sync()
    res = ahf.results_to_numpy(out["res"])
    bound = out["bound_idx"].cpu().numpy()
    phi = out["phi"].cpu().numpy()
    rem = out["removed_iter"].cpu().numpy()
    prof = out["prof"].cpu().numpy()

    # every size class is present, and every halo is compared
    assert len(_sample(pop.count)) >= 25
    s = compare(pop, prm, res, bound, phi, rem)
    assert s["halos"] == 2000
    check_profiles(pop, prm, res, prof, N_BINS, R_MIN_FRAC)

    # every halo: record invariants and consistency of the per-slot outputs
    crit = prm.delta_rho * 4.0 * math.pi / 3.0
    assert np.all(res["n_bound"] <= res["n_member"]) and np.all(res["n_member"] <= pop.count)
    assert int(res["part_iter"].sum()) == 6_017_597
    for h in range(pop.n_halos):
        r = res[h]
        lo, n, nb = int(pop.offset[h]), int(pop.count[h]), int(r["n_bound"])
        seg = rem[lo:lo + n]
        assert int(np.sum(seg == 0)) == nb
        assert int(np.sum(seg >= 0)) == int(r["n_member"])
        assert r["status"] & ahf.HALO_NOT_CONVERGED == 0
        b = bound[lo:lo + nb]
        assert np.all((b >= lo) & (b < lo + n)) and np.all(rem[b] == 0)
        if r["r_vir"] > 0:
            # Eq. 1 holds exactly at r_vir by construction (M_vir / (4/3 pi r_vir^3))
            assert abs(r["m_vir"] / (crit * r["r_vir"] ** 3) - 1.0) < 1e-12
            # the rows' last cumulative mass is M(<= r_vir) = M_vir
            assert prof[h, -1, 1] == pytest.approx(r["m_vir"], rel=1e-12)
        # phi rises outwards along the bound list (within float rounding)
        ph = phi[lo:lo + nb].astype(np.float64)
        assert np.all(np.diff(ph) >= -1e-6 * np.abs(ph[1:]))

"""CUDA path vs the CPU oracle, element by element (through the C ABI)."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import run_gpu
from tests.parity import compare

pytestmark = pytest.mark.gpu


def test_onchip_batch_f32_rel():
    # all three on-chip variants, several tiles, ragged sizes
    pop = synth.halo_batch(seed=7, n_halos=60, n_lo=100, n_hi=7000)
    assert pop.count.max() <= 8192
    out, prm, _, _ = run_gpu(pop)
    s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    assert s["halos"] == 60


def test_onchip_batch_f64_multimass():
    pop = synth.halo_batch(seed=8, n_halos=30, n_lo=100, n_hi=5000, coord_type=synth.COORD_F64,
                           with_masses=True)
    out, prm, _, _ = run_gpu(pop)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])


def test_single_nfw_halo_f64():
    # one 10k-particle NFW halo + 1k background, float64 (multi-CTA class)
    pop = synth.single_halo()
    out, prm, _, _ = run_gpu(pop)
    s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    assert out["res"][0]["n_bound"] > 9000


def test_multi_cta_class_forced_small():
    # route every halo above 1024 candidates through the multi-CTA class
    from paper_0904_3662_gb300 import ahf
    from tests.gpu_util import require_gpu
    require_gpu()
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_ONCHIP_MAX, 1024)
    pop = synth.halo_batch(seed=9, n_halos=25, n_lo=300, n_hi=30000)
    out, prm, _, _ = run_gpu(pop, ctx=ctx)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])


def test_multi_cta_class_f64_masses():
    from paper_0904_3662_gb300 import ahf
    from tests.gpu_util import require_gpu
    require_gpu()
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_ONCHIP_MAX, 0)
    pop = synth.halo_batch(seed=10, n_halos=12, n_lo=100, n_hi=9000, coord_type=synth.COORD_F64,
                           with_masses=True)
    out, prm, _, _ = run_gpu(pop, ctx=ctx)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])


def test_cluster_variants_all_sizes():
    # haloes of 8k..125k candidates: clusters of 2, 4, 8 and 16 CTAs, at and
    # around every class boundary
    rng = np.random.default_rng(31)
    from tests.test_gpu_paths import _pop_from_arrays
    pl, vl, cs, rs = [], [], [], []
    for n in (8193, 9000, 16384, 16385, 20000, 32768, 32769, 50000, 65536, 65537, 90000, 125000):
        n_nfw = int(n * 0.87)
        p, v = synth.sample_nfw(rng, n_nfw, 10.0, 150.0)
        p2, v2 = synth.sample_uniform_sphere(rng, n - n_nfw, 300.0, 600.0)
        pl.append(np.concatenate([p, p2])); vl.append(np.concatenate([v, v2]))
        cs.append([0.0, 0.0, 0.0]); rs.append(300.0)
    pop = _pop_from_arrays(pl, vl, cs, rs, m0=synth.PARTICLE_MASS)
    out, prm, ctx, _ = run_gpu(pop)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    st = ctx.stats()
    assert st["phase_halos"][4:8] == [3, 3, 3, 3], st


def test_cluster_and_grid_agree_bitwise():
    # the same haloes through clusters and through the multi-CTA class
    from paper_0904_3662_gb300 import ahf
    from tests.gpu_util import require_gpu
    require_gpu()
    pop = synth.halo_batch(seed=32, n_halos=8, n_lo=9000, n_hi=60000)
    a, prm, ctx, _ = run_gpu(pop)
    ctx2 = ahf.Context(0)
    ctx2.set_option(ahf.OPT_ONCHIP_MAX, 0)
    b, _, _, _ = run_gpu(pop, ctx=ctx2)
    np.testing.assert_array_equal(a["removed_iter"], b["removed_iter"])
    np.testing.assert_array_equal(a["res"].view(np.uint8), b["res"].view(np.uint8))
    for h in range(pop.n_halos):
        lo, nb = int(pop.offset[h]), int(a["res"][h]["n_bound"])
        np.testing.assert_array_equal(a["bound_idx"][lo:lo + nb], b["bound_idx"][lo:lo + nb])
        np.testing.assert_array_equal(a["phi"][lo:lo + nb], b["phi"][lo:lo + nb])


def test_all_fp64_mode_single_and_batch():
    # the all-FP64 path: phi to 1e-11, virial to 1e-11, bound lists in the
    # oracle's exact radial order
    from paper_0904_3662_gb300 import ahf
    from tests.gpu_util import require_gpu
    require_gpu()
    for pop in (synth.single_halo(),
                synth.halo_batch(seed=51, n_halos=25, n_lo=100, n_hi=20000, coord_type=synth.COORD_F64,
                                 with_masses=True),
                synth.halo_batch(seed=52, n_halos=10, n_lo=100, n_hi=5000)):
        prm = ahf.params_for(pop, precision=ahf.PREC_FP64)
        out, prm, ctx, _ = run_gpu(pop, params=prm)
        assert out["phi"].dtype == np.float64
        s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=1e-11,
                    vir_rtol=1e-11, exact_order=True)
        assert s["worst_phi_rel"] < 1e-11


def test_all_fp64_mode_periodic_box():
    from paper_0904_3662_gb300 import ahf
    from tests.gpu_util import require_gpu
    require_gpu()
    pop = synth.large_tail(seed=53, n_halos=2, n_lo=3000, n_hi=20000, n_sub=4, box=5e5)
    prm = ahf.params_for(pop, precision=ahf.PREC_FP64)
    out, prm, _, _ = run_gpu(pop, params=prm)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=1e-11,
            vir_rtol=1e-11, exact_order=True)

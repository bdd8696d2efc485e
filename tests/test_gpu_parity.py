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

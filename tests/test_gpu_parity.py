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

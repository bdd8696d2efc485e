"""The autotuner's knobs change the time, never the results: every routing
of haloes to size classes, the promotion rule and the pass chunk give the
same bits (the sums are exact fixed point).  The tuning file is applied by
ahf_create only for its own device and build; a short search runs."""
import os

import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _run(ahf, torch, pop, options):
    ctx = ahf.Context(0)
    for opt, val in options.items():
        ctx.set_option(opt, val)
    parts = ahf.particles_from_population(pop)
    out = ctx.unbind_batch(parts, ahf.halos_from_population(pop), ahf.params_for(pop))
    torch.cuda.synchronize()
    ctx.sync()
    return (ahf.results_to_numpy(out["res"]), out["bound_idx"].cpu().numpy(), out["phi"].cpu().numpy(),
            out["removed_iter"].cpu().numpy(), ctx.stats())


def test_every_tuned_configuration_gives_the_same_bits():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=61, n_halos=50, n_lo=100, n_hi=200_000)
    assert pop.count.max() > 40_000          # the fourth setting routes it to the multi-CTA class
    caps = ahf.VARIANT_CAPS
    configs = [
        {},
        {ahf.OPT_PROMOTE: 0},
        {ahf.OPT_PROMOTE: 0, **{ahf.OPT_CLASS_CUT + v: caps[v] // 2 for v in range(7)}},
        {ahf.OPT_CLASS_CUT + 7: 40_000, ahf.OPT_PASS_CHUNK: 1},    # more haloes in the multi-CTA class
        {ahf.OPT_CLASS_CUT + 2: 0, ahf.OPT_CLASS_CUT + 5: 0, ahf.OPT_PASS_CHUNK: 16},
    ]
    ref = _run(ahf, torch, pop, configs[0])
    res0, b0, p0, r0, _ = ref
    classes = set()
    for cfg in configs[1:]:
        res, b, p, r, st = _run(ahf, torch, pop, cfg)
        classes |= {k for k in range(ahf.N_PHASES) if st["phase_halos"][k] > 0}
        assert res.tobytes() == res0.tobytes(), cfg
        np.testing.assert_array_equal(r, r0)
        for h in range(pop.n_halos):
            lo, nb = int(pop.offset[h]), int(res0["n_bound"][h])
            np.testing.assert_array_equal(b[lo:lo + nb], b0[lo:lo + nb])
            assert p[lo:lo + nb].tobytes() == p0[lo:lo + nb].tobytes()
    assert ahf.PHASE_NAMES.index("grid_gather_sort") in classes


def test_tuning_file_applies_only_to_its_device_and_build(tmp_path, monkeypatch):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf, autotune
    key = autotune.device_key(torch.cuda.get_device_name(0))
    p = str(tmp_path / "tune.txt")
    autotune.write(p, key, ahf.build_id(), {ahf.OPT_PROMOTE: 0, ahf.OPT_CLASS_CUT + 1: 700, ahf.OPT_PASS_CHUNK: 4})
    monkeypatch.setenv("AHF_TUNING", p)
    ctx = ahf.Context(0)
    assert ctx.get_option(ahf.OPT_PROMOTE) == 0
    assert ctx.get_option(ahf.OPT_CLASS_CUT + 1) == 700
    assert ctx.get_option(ahf.OPT_PASS_CHUNK) == 4
    ctx.set_option(ahf.OPT_PASS_CHUNK, 8)                 # set_option still overrides
    assert ctx.get_option(ahf.OPT_PASS_CHUNK) == 8
    # another build: ignored
    autotune.write(p, key, "0000000000000000", {ahf.OPT_PROMOTE: 0})
    assert ahf.Context(0).get_option(ahf.OPT_PROMOTE) == 1
    # a file that does not parse: an error
    with open(p, "w") as f:
        f.write("nonsense\n")
    with pytest.raises(ahf.AHFError):
        ahf.Context(0)


def test_a_short_search_returns_a_configuration_no_slower():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf, autotune
    pop = synth.halo_batch(seed=62, n_halos=300, n_lo=100, n_hi=20_000)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    out = ctx.alloc_outputs(pop.n_halos, pop.n_particles)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def step():
        ctx.unbind_batch(parts, hal, prm, out=out)

    cfg, default, best, trials = autotune.tune(ctx, step, ahf, False, flush, reps=3, sweeps=1, budget_s=15.0)
    assert best <= default and len(trials) >= 2
    assert set(cfg) == {o for o, _ in autotune.knobs(ahf, False)}

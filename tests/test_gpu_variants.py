"""Method variants on the GPU against the oracle: the bulk velocity fixed
from the initial set (every class), the second pass within r_vir, the
subhalo edge at the rise of the density profile, gas thermal energy."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu
from tests.parity import check_profiles, compare

pytestmark = pytest.mark.gpu


def _prm(pop, variant, **kw):
    from paper_0904_3662_gb300 import ahf
    return ahf.params_for(pop, variant=variant, **kw)


def test_initial_bulk_velocity_hand_case():
    from paper_0904_3662_gb300 import ahf
    from tests.test_gpu_paths import _pop_from_arrays
    require_gpu()
    pos = np.array([[1.0, 0, 0], [50.0, 0, 0], [100.0, 0, 0]])
    vel = np.array([[0.0, 0, 0], [3000.0, 0, 0], [600.0, 0, 0]])
    pop = _pop_from_arrays([pos], [vel], [[0, 0, 0]], [200.0], coord_type=synth.COORD_F64,
                           masses=[np.array([1e12, 2e11, 1e9])])
    for variant, want in ((0, [0, 1, 2]), (ahf.VAR_VBULK_INITIAL, [0, 1, 0])):
        out, prm, _, _ = run_gpu(pop, params=_prm(pop, variant, H=0.0))
        assert out["removed_iter"].tolist() == want, variant


@pytest.mark.parametrize("onchip_max", [None, 0])
def test_initial_bulk_velocity_every_class(onchip_max):
    from paper_0904_3662_gb300 import ahf
    require_gpu()
    pop = synth.halo_batch(seed=92, n_halos=40, n_lo=100, n_hi=100_000)
    ctx = ahf.Context(0)
    if onchip_max is not None:
        ctx.set_option(ahf.OPT_ONCHIP_MAX, onchip_max)          # everything through the multi-CTA class
    out, prm, _, _ = run_gpu(pop, params=_prm(pop, ahf.VAR_VBULK_INITIAL), ctx=ctx)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    base, _, _, _ = run_gpu(pop, ctx=ctx)
    assert not np.array_equal(base["removed_iter"], out["removed_iter"])      # the variant matters here


def test_retruncation_batch_with_profile_and_host_entry():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=93, n_halos=40, n_lo=100, n_hi=60_000)
    prm = _prm(pop, ahf.VAR_RETRUNCATE)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    out = ctx.unbind_profile_batch(parts, hal, prm, n_bins=16, r_min_frac=0.02)
    torch.cuda.synchronize()
    ctx.sync()
    res = ahf.results_to_numpy(out["res"])
    host = {k: out[k].cpu().numpy() for k in ("bound_idx", "phi", "removed_iter", "prof")}
    compare(pop, prm, res, host["bound_idx"], host["phi"], host["removed_iter"])
    check_profiles(pop, prm, res, host["prof"], 16, 0.02)
    # the same through host buffers
    hp = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, pop.m0, pop.coord_type)
    h = ctx.unbind_batch_host(hp, hal, prm, n_bins=16, r_min_frac=0.02)
    assert h["res"].tobytes() == res.tobytes()
    np.testing.assert_array_equal(h["removed_iter"], host["removed_iter"])
    # a second pass never keeps more than the first
    one, _, _, _ = run_gpu(pop, ctx=ctx)
    assert np.all(res["n_bound"] <= one["res"]["n_bound"])


def test_variant_arguments_checked():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=94, n_halos=3, n_lo=100, n_hi=500)
    with pytest.raises(ahf.AHFError) as e:
        run_gpu(pop, params=_prm(pop, ahf.VAR_RETRUNCATE), plain=True)
    assert e.value.code == ahf.ERR_INVALID
    with pytest.raises(ahf.AHFError):
        run_gpu(pop, params=_prm(pop, 8))                       # unknown bit


@pytest.mark.parametrize("coord_type,precision", [(synth.COORD_F32_REL, 0), (synth.COORD_F64, 1)])
def test_gas_thermal_energy(coord_type, precision):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    base = synth.halo_batch(seed=96, n_halos=25, n_lo=100, n_hi=30_000, coord_type=coord_type)
    pop = synth.with_gas(base, frac=0.3)
    prm = ahf.params_for(pop, precision=precision)
    tol = 1e-11 if precision else 1e-5
    out, prm, ctx, _ = run_gpu(pop, params=prm)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=tol,
            vir_rtol=max(tol, 1e-5), exact_order=bool(precision))
    st = ctx.stats()
    assert st["phase_halos"][8] == pop.n_halos                  # gas runs in the multi-CTA class
    # the thermal energy removes particles the collisionless run keeps
    cold, _, _, _ = run_gpu(base, params=ahf.params_for(base, precision=precision), ctx=ctx)
    assert np.all(out["res"]["n_bound"] <= cold["res"]["n_bound"])
    assert np.any(out["res"]["n_bound"] < cold["res"]["n_bound"])
    # the plain path and the host entry agree with the batch
    plain, _, _, _ = run_gpu(pop, params=prm, ctx=ctx, plain=True)
    assert plain["res"].tobytes() == out["res"].tobytes()
    hp = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, pop.m0, pop.coord_type, pop.u_th)
    h = ctx.unbind_batch_host(hp, ahf.halos_from_population(pop), prm)
    assert h["res"].tobytes() == out["res"].tobytes()


@pytest.mark.parametrize("onchip_max", [None, 0])
def test_rise_edge_every_class(onchip_max):
    # designed profiles of 400, 1,600 and 20,000 particles (warp, one CTA,
    # 2-CTA cluster; or all in the multi-CTA class) end at the last particle
    # of shell 11; a falling profile keeps its edge; records, bound lists and
    # profile rows against the oracle
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    for rise in (True, False):
        pop = synth.shell_profile_batch(rise=rise)
        ctx = ahf.Context(0)
        ctx.set_option(ahf.OPT_PROMOTE, 0)
        if onchip_max is not None:
            ctx.set_option(ahf.OPT_ONCHIP_MAX, onchip_max)
        prm = _prm(pop, ahf.VAR_RISE_EDGE)
        out, prm, _, _ = run_gpu(pop, params=prm, ctx=ctx)
        compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
        res = out["res"]
        for h in range(pop.n_halos):
            n = int(pop.count[h]) // 16
            if rise:
                assert res[h]["status"] == ahf.HALO_RVIR_BEYOND_EDGE | ahf.HALO_RISE_EDGE
                assert res[h]["k_vir"] == 12 * n - 1
            else:
                assert res[h]["status"] == ahf.HALO_RVIR_BEYOND_EDGE
        parts = ahf.particles_from_population(pop)
        p2 = ctx.unbind_profile_batch(parts, ahf.halos_from_population(pop), prm, n_bins=16, r_min_frac=0.05)
        torch.cuda.synchronize()
        r2 = ahf.results_to_numpy(p2["res"])
        assert r2.tobytes() == res.tobytes()
        check_profiles(pop, prm, r2, p2["prof"].cpu().numpy(), 16, 0.05)

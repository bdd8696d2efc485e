"""GPU: every entry point of the C ABI against the oracle, plus the edge cases
of the method (empty, ragged, degenerate haloes)."""
import copy
import math

import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu
from tests.parity import check_profiles as _check_profiles, compare, oracle_params

pytestmark = pytest.mark.gpu


def _pop_from_arrays(pos_list, vel_list, centres, radii, coord_type=synth.COORD_F32_REL, masses=None, m0=1e9,
                     box=0.0):
    """A population from explicit per-halo arrays (candidates back to back)."""
    counts = np.array([p.shape[0] for p in pos_list], dtype=np.int64)
    offset = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    pos = np.concatenate(pos_list) if counts.sum() else np.zeros((0, 3))
    vel = np.concatenate(vel_list) if counts.sum() else np.zeros((0, 3))
    dt = np.float64 if coord_type == synth.COORD_F64 else np.float32
    m = None if masses is None else np.concatenate(masses).astype(dt)
    return synth.Population(
        name="custom", coord_type=coord_type,
        x=pos[:, 0].astype(dt), y=pos[:, 1].astype(dt), z=pos[:, 2].astype(dt),
        vx=vel[:, 0].astype(dt), vy=vel[:, 1].astype(dt), vz=vel[:, 2].astype(dt),
        m=m, m0=m0, box=box, centre=np.asarray(centres, dtype=np.float64).reshape(-1, 3),
        radius=np.asarray(radii, dtype=np.float64), offset=offset, count=counts,
        r200=np.zeros(len(counts)), conc=np.zeros(len(counts)))


def _check_all(pop, ctx=None, **kw):
    out, prm, ctx, dev = run_gpu(pop, ctx=ctx, **kw)
    s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    return out, prm, ctx, dev, s


def test_edge_cases_small():
    rng = np.random.default_rng(1)
    pl, vl, cs, rs = [], [], [], []
    # 0: empty halo
    pl.append(np.zeros((0, 3))); vl.append(np.zeros((0, 3))); cs.append([0, 0, 0]); rs.append(10.0)
    # 1: single particle (Hubble flow unbinds it)
    pl.append(np.array([[3.0, 0, 0]])); vl.append(np.array([[10.0, 0, 0]])); cs.append([0, 0, 0]); rs.append(10.0)
    # 2: nobody inside the gather sphere
    pl.append(rng.uniform(50, 60, (20, 3))); vl.append(np.zeros((20, 3))); cs.append([0, 0, 0]); rs.append(1.0)
    # 3: a particle exactly at the centre plus a bound cloud
    p, v = synth.sample_uniform_sphere(rng, 300, 5.0, 20.0)
    p[0] = 0.0
    pl.append(p); vl.append(v); cs.append([0, 0, 0]); rs.append(10.0)
    # 4: duplicate positions (radius ties)
    p, v = synth.sample_uniform_sphere(rng, 200, 5.0, 20.0)
    p[100:150] = p[0:50]
    pl.append(p); vl.append(v); cs.append([0, 0, 0]); rs.append(10.0)
    # 5: every particle at 10 v_esc: all removed (EMPTY)
    p, _ = synth.sample_uniform_sphere(rng, 500, 5.0, 0.0)
    d = rng.standard_normal((500, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    vl.append(d * 3000.0); pl.append(p); cs.append([0, 0, 0]); rs.append(10.0)
    # 6: cold sphere moving with the bulk (nothing removed without Hubble flow in its frame)
    p, _ = synth.sample_uniform_sphere(rng, 700, 5.0, 0.0)
    pl.append(p); vl.append(np.tile([[300.0, -200.0, 50.0]], (700, 1))); cs.append([0, 0, 0]); rs.append(10.0)
    # 7, 8: every member at one radius (axis points: the float radius is exact),
    # with non-members outside the sphere; the sort's key range is then only
    # the step between members and non-members
    for n_axis, n_out in ((60, 10), (700, 100)):
        ax = np.repeat(np.vstack([np.eye(3), -np.eye(3)]) * 4.0, n_axis // 6 + 1, axis=0)[:n_axis]
        p = np.vstack([ax, rng.uniform(40, 50, (n_out, 3))])
        pl.append(p); vl.append(rng.normal(0, 5.0, p.shape)); cs.append([0, 0, 0]); rs.append(10.0)
    # ragged sizes just around the class boundaries
    for n in (31, 32, 33, 511, 512, 513, 1023, 1024, 1025, 4095, 4097, 8191, 8192):
        p, v = synth.sample_nfw(rng, n, 10.0, 60.0)
        pl.append(p); vl.append(v); cs.append([0, 0, 0]); rs.append(120.0)
    pop = _pop_from_arrays(pl, vl, cs, rs, m0=1e9)
    out, prm, ctx, dev, s = _check_all(pop)
    res = out["res"]
    assert res[0]["status"] & O.EMPTY and res[0]["n_iter"] == 0
    assert res[2]["n_member"] == 0 and res[2]["status"] & O.EMPTY
    assert res[5]["status"] & O.EMPTY
    assert (out["removed_iter"][int(pop.offset[2]):int(pop.offset[2]) + 20] == -1).all()
    assert res[7]["n_member"] == 60 and res[8]["n_member"] == 700


def test_edge_cases_multi_cta():
    # the same degenerate haloes through the multi-CTA class
    from paper_0904_3662_gb300 import ahf
    require_gpu()
    rng = np.random.default_rng(2)
    pl, vl, cs, rs = [], [], [], []
    pl.append(np.zeros((0, 3))); vl.append(np.zeros((0, 3))); cs.append([0, 0, 0]); rs.append(10.0)
    pl.append(np.array([[3.0, 0, 0]])); vl.append(np.array([[10.0, 0, 0]])); cs.append([0, 0, 0]); rs.append(10.0)
    pl.append(rng.uniform(50, 60, (20, 3))); vl.append(np.zeros((20, 3))); cs.append([0, 0, 0]); rs.append(1.0)
    p, v = synth.sample_uniform_sphere(rng, 3000, 5.0, 20.0)
    p[0] = 0.0
    p[1500:2000] = p[0:500]
    pl.append(p); vl.append(v); cs.append([0, 0, 0]); rs.append(10.0)
    p, _ = synth.sample_uniform_sphere(rng, 2500, 5.0, 0.0)
    d = rng.standard_normal((2500, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pl.append(p); vl.append(d * 3000.0); cs.append([0, 0, 0]); rs.append(10.0)
    for n in (2047, 2048, 2049, 6000):
        p, v = synth.sample_nfw(rng, n, 10.0, 60.0)
        pl.append(p); vl.append(v); cs.append([0, 0, 0]); rs.append(120.0)
    pop = _pop_from_arrays(pl, vl, cs, rs, m0=1e9)
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_ONCHIP_MAX, 0)
    _check_all(pop, ctx=ctx)


def test_member_index_list_and_gather_radius():
    # candidates given through a permuted member list; gather radius cuts
    # part of each halo
    pop = synth.halo_batch(seed=11, n_halos=15, n_lo=200, n_hi=12000)
    rng = np.random.default_rng(0)
    perm = rng.permutation(pop.n_particles).astype(np.int64)
    # member slots: halo h's slice lists its particles in shuffled order
    member = np.empty(pop.n_particles, dtype=np.int64)
    for h in range(pop.n_halos):
        lo, n = int(pop.offset[h]), int(pop.count[h])
        member[lo:lo + n] = lo + rng.permutation(n)
    q = copy.copy(pop)
    q.radius = pop.radius * 0.6
    out, prm, _, _ = run_gpu(q, member_idx=member)
    compare(q, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], member_idx=member)


@pytest.mark.parametrize("n_lo,n_hi", [(1500, 6000), (20_000, 40_000)])
def test_periodic_box_float32_coordinates(n_lo, n_hi):
    # haloes straddling the edges of a periodic box, float32 box coordinates
    # (on-chip and multi-CTA classes)
    pop = synth.large_tail(seed=5, n_halos=3, n_lo=n_lo, n_hi=n_hi, n_sub=5, box=5e5)
    pop.centre[0] = [10.0, 499_990.0, 250_000.0]
    pop.centre[1] = [499_999.0, 5.0, 3.0]
    # rebuild coordinates around the moved centres
    src = synth.large_tail(seed=5, n_halos=3, n_lo=n_lo, n_hi=n_hi, n_sub=5, box=5e5)
    for h in range(2):
        s = slice(int(pop.offset[h]), int(pop.offset[h] + pop.count[h]))
        for a, k in enumerate("xyz"):
            rel = getattr(src, k)[s].astype(np.float64) - src.centre[h, a]
            rel = (rel + 2.5e5) % 5e5 - 2.5e5
            getattr(pop, k)[s] = np.mod(rel + pop.centre[h, a], 5e5).astype(np.float32)
    out, prm, _, _ = run_gpu(pop)
    s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    assert all(out["res"][h]["n_bound"] > 0.5 * pop.count[h] for h in range(3))


def test_not_converged_and_softening():
    pop = synth.halo_batch(seed=12, n_halos=10, n_lo=300, n_hi=20000)
    from paper_0904_3662_gb300 import ahf
    prm = ahf.params_for(pop, max_iter=1, r_soft=0.5)
    out, prm, _, _ = run_gpu(pop, params=prm)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    assert any(r["status"] & O.NOT_CONVERGED for r in out["res"])


def test_plain_path_matches_batched():
    pop = synth.halo_batch(seed=13, n_halos=12, n_lo=100, n_hi=15000)
    a, prm, ctx, _ = run_gpu(pop)
    b, _, _, _ = run_gpu(pop, plain=True, ctx=ctx)
    compare(pop, prm, b["res"], b["bound_idx"], b["phi"], b["removed_iter"])
    for h in range(pop.n_halos):
        nb = int(a["res"][h]["n_bound"])
        lo = int(pop.offset[h])
        assert int(b["res"][h]["n_bound"]) == nb
        np.testing.assert_array_equal(np.sort(a["bound_idx"][lo:lo + nb]), np.sort(b["bound_idx"][lo:lo + nb]))


def test_host_entry_point_with_profile():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=14, n_halos=20, n_lo=100, n_hi=12000)
    ctx = ahf.Context(0)
    parts = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, pop.m0, pop.coord_type)
    prm = ahf.params_for(pop)
    out = ctx.unbind_batch_host(parts, ahf.halos_from_population(pop), prm, n_bins=16, r_min_frac=0.02)
    compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"])
    _check_profiles(pop, prm, out["res"], out["prof"], 16, 0.02)


def _pinned(torch, a):
    """A page-locked copy of a numpy array (same dtype and shape)."""
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.reshape(-1).view(np.uint8)).pin_memory()
    return t, t.numpy().view(a.dtype).reshape(a.shape)


def test_host_entry_point_pushes_under_graph_replay():
    # the host-buffer call with its outputs pushed per size class, as a
    # replayed CUDA graph: a second call on the same buffers replays the
    # captured graph (its outputs zeroed before, so a replay that pushed
    # nothing would show), a call on other output buffers captures anew; every
    # call's results equal the device entry point's
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=17, n_halos=60, n_lo=100, n_hi=20000)
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_GRAPHS, 1)
    ctx.set_option(ahf.OPT_HOST_DIRECT, 2)
    keep = []

    def pin(a):
        t, v = _pinned(torch, a)
        keep.append(t)
        return v
    parts = ahf.Particles(pin(pop.x), pin(pop.y), pin(pop.z), pin(pop.vx), pin(pop.vy), pin(pop.vz), None,
                          pop.m0, pop.coord_type)
    prm = ahf.params_for(pop)
    hal = ahf.halos_from_population(pop)
    n = pop.n_particles

    def buffers():
        return {"res": pin(np.zeros(pop.n_halos, dtype=ahf.RESULT_DTYPE)), "bound_idx": pin(np.zeros(n, np.int64)),
                "phi": pin(np.zeros(n, np.float32)), "removed_iter": pin(np.zeros(n, np.int32)),
                "prof": pin(np.zeros((pop.n_halos, 16, 4)))}
    a, b = buffers(), buffers()
    got, graphs = [], []
    for out in (a, a, b):
        for v in out.values():
            v[...] = 0
        ctx.unbind_batch_host(parts, hal, prm, out=out, n_bins=16, r_min_frac=0.02)
        st = ctx.stats()
        graphs.append((st["graph_captures"], st["graph_launches"]))
        got.append({k: v.copy() for k, v in out.items()})
    assert graphs == [(1, 1), (0, 1), (1, 1)]
    dev = ctx.unbind_profile_batch(ahf.particles_from_population(pop), hal, prm, n_bins=16, r_min_frac=0.02)
    torch.cuda.synchronize()
    res_d = ahf.results_to_numpy(dev["res"])
    bi_d, phi_d = dev["bound_idx"].cpu().numpy(), dev["phi"].cpu().numpy()
    for o in got:
        assert o["res"].tobytes() == res_d.tobytes()
        np.testing.assert_array_equal(o["removed_iter"], dev["removed_iter"].cpu().numpy())
        np.testing.assert_array_equal(o["prof"], dev["prof"].cpu().numpy())
        for h in range(pop.n_halos):
            lo, nb = int(pop.offset[h]), int(res_d[h]["n_bound"])
            np.testing.assert_array_equal(o["bound_idx"][lo:lo + nb], bi_d[lo:lo + nb])
            np.testing.assert_array_equal(o["phi"][lo:lo + nb], phi_d[lo:lo + nb])


@pytest.mark.parametrize("onchip_max", [131072, 8192])
def test_host_entry_point_page_locked_in_place_and_staged(onchip_max):
    # page-locked inputs and outputs used in place by the kernels (1), the
    # inputs read in place with the outputs pushed by each class as it
    # finishes (2), against the staged route (0) and the device entry point:
    # identical results; with the on-chip classes capped at 8,192 candidates
    # the larger haloes take the multi-CTA class (its push after its kernels)
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=16, n_halos=40, n_lo=100, n_hi=40000, with_masses=True)
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_ONCHIP_MAX, onchip_max)
    keep = []

    def pin(a):
        t, v = _pinned(torch, a)
        keep.append(t)
        return v
    parts = ahf.Particles(pin(pop.x), pin(pop.y), pin(pop.z), pin(pop.vx), pin(pop.vy), pin(pop.vz), pin(pop.m),
                          pop.m0, pop.coord_type)
    prm = ahf.params_for(pop)
    hal = ahf.halos_from_population(pop)
    n = pop.n_particles
    outs = []
    for direct in (2, 1, 0):
        ctx.set_option(ahf.OPT_HOST_DIRECT, direct)
        assert ctx.get_option(ahf.OPT_HOST_DIRECT) == direct
        out = {"res": pin(np.zeros(pop.n_halos, dtype=ahf.RESULT_DTYPE)), "bound_idx": pin(np.zeros(n, np.int64)),
               "phi": pin(np.zeros(n, np.float32)), "removed_iter": pin(np.zeros(n, np.int32)),
               "prof": pin(np.zeros((pop.n_halos, 16, 4)))}
        ctx.unbind_batch_host(parts, hal, prm, out=out, n_bins=16, r_min_frac=0.02)
        outs.append({k: v.copy() for k, v in out.items()})
    dev = ctx.unbind_profile_batch(ahf.particles_from_population(pop), hal, prm, n_bins=16, r_min_frac=0.02)
    torch.cuda.synchronize()
    st = ctx.stats()
    if onchip_max < 40000:
        assert st["phase_halos"][ahf.PHASE_NAMES.index("grid_gather_sort")] > 0
    res_d = ahf.results_to_numpy(dev["res"])
    for o in outs:
        assert o["res"].tobytes() == res_d.tobytes()
        np.testing.assert_array_equal(o["removed_iter"], dev["removed_iter"].cpu().numpy())
        np.testing.assert_array_equal(o["prof"], dev["prof"].cpu().numpy())
        for h in range(pop.n_halos):
            lo, nb = int(pop.offset[h]), int(res_d["n_bound"][h])
            np.testing.assert_array_equal(o["bound_idx"][lo:lo + nb], dev["bound_idx"].cpu().numpy()[lo:lo + nb])
            np.testing.assert_array_equal(o["phi"][lo:lo + nb], dev["phi"].cpu().numpy()[lo:lo + nb])
    compare(pop, prm, outs[0]["res"], outs[0]["bound_idx"], outs[0]["phi"], outs[0]["removed_iter"])


def test_profile_batch_device():
    torch = require_gpu()
    pop = synth.halo_batch(seed=15, n_halos=30, n_lo=100, n_hi=20000, with_masses=True)
    out, prm, ctx, dev = run_gpu(pop)
    from paper_0904_3662_gb300 import ahf
    parts = ahf.particles_from_population(pop)
    prof = ctx.profile_batch(parts, ahf.halos_from_population(pop), prm, dev["res"], dev["bound_idx"], n_bins=24,
                             r_min_frac=0.01)
    torch.cuda.synchronize()
    _check_profiles(pop, prm, out["res"], prof.cpu().numpy(), 24, 0.01)


def test_bitwise_repeatable_and_batch_independent():
    # exact sums: identical outputs run to run and alone vs in a batch
    torch = require_gpu()
    pop = synth.halo_batch(seed=16, n_halos=40, n_lo=100, n_hi=20000)
    a, prm, ctx, _ = run_gpu(pop)
    b, _, _, _ = run_gpu(pop, ctx=ctx)
    np.testing.assert_array_equal(a["removed_iter"], b["removed_iter"])
    np.testing.assert_array_equal(a["res"].view(np.uint8), b["res"].view(np.uint8))
    for h in range(pop.n_halos):          # slots past n_bound are unspecified
        lo, nb = int(pop.offset[h]), int(a["res"][h]["n_bound"])
        np.testing.assert_array_equal(a["bound_idx"][lo:lo + nb], b["bound_idx"][lo:lo + nb])
        np.testing.assert_array_equal(a["phi"][lo:lo + nb], b["phi"][lo:lo + nb])
    # halo 3 alone
    h = 3
    one = copy.copy(pop)
    for k in ("centre", "radius", "offset", "count", "r200", "conc"):
        setattr(one, k, getattr(pop, k)[h:h + 1])
    c, _, _, _ = run_gpu(one, ctx=ctx)
    lo, nb = int(pop.offset[h]), int(a["res"][h]["n_bound"])
    np.testing.assert_array_equal(c["bound_idx"][lo:lo + nb], a["bound_idx"][lo:lo + nb])
    np.testing.assert_array_equal(c["phi"][lo:lo + nb], a["phi"][lo:lo + nb])
    assert c["res"][0].tobytes() == a["res"][h].tobytes()


def test_invalid_arguments_are_rejected():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=17, n_halos=3, n_lo=100, n_hi=500)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    bad = hal.copy()
    bad["offset"][1] = bad["offset"][0]          # shared slots
    with pytest.raises(ahf.AHFError) as e:
        ctx.unbind_batch(parts, bad, ahf.params_for(pop))
    assert e.value.code == ahf.ERR_INVALID
    bad = hal.copy()
    bad["count"][2] += 10 ** 9                   # beyond the particle store
    with pytest.raises(ahf.AHFError):
        ctx.unbind_batch(parts, bad, ahf.params_for(pop))
    with pytest.raises(ahf.AHFError):
        ctx.unbind_batch(parts, hal, ahf.params_for(pop, max_iter=0))
    with pytest.raises(ahf.AHFError):
        ctx.set_option(ahf.OPT_ONCHIP_MAX, 10 ** 7)
    # out-of-range member index: reported by ahf_sync, no fault
    import torch
    member = torch.arange(pop.n_particles, dtype=torch.int64, device="cuda")
    member[5] = 10 ** 12
    ctx.unbind_batch(parts, hal, ahf.params_for(pop), member_idx=member)
    with pytest.raises(ahf.AHFError) as e:
        ctx.sync()
    assert e.value.code == ahf.ERR_INVALID
    ctx.sync()                                    # cleared


@pytest.mark.parametrize("with_masses", [True, False])
def test_fused_profile_matches_standalone_and_oracle(with_masses):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    # every class: warp, CTA, clusters (and the multi-CTA class through a second context)
    pop = synth.halo_batch(seed=41, n_halos=60, n_lo=100, n_hi=100_000, with_masses=with_masses)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    for onchip_max in (None, 0):
        if onchip_max is not None:
            ctx.set_option(ahf.OPT_ONCHIP_MAX, onchip_max)
        fused = ctx.unbind_profile_batch(parts, hal, prm, n_bins=20, r_min_frac=0.02)
        sep = ctx.profile_batch(parts, hal, prm, fused["res"], fused["bound_idx"], n_bins=20, r_min_frac=0.02)
        torch.cuda.synchronize()
        a = fused["prof"].cpu().numpy()
        b = sep.cpu().numpy()
        np.testing.assert_array_equal(a[:, :, 0], b[:, :, 0])
        np.testing.assert_allclose(a[:, :, 1], b[:, :, 1], rtol=1e-12, atol=0)
        # density and v_circ are formed in float from the (exact) masses
        np.testing.assert_allclose(a[:, :, 2:], b[:, :, 2:], rtol=1e-6, atol=0)
        res = ahf.results_to_numpy(fused["res"])
        compare(pop, prm, res, fused["bound_idx"].cpu().numpy(), fused["phi"].cpu().numpy(),
                fused["removed_iter"].cpu().numpy())
        _check_profiles(pop, prm, res, a, 20, 0.02)


def test_graph_replay_matches_plain_launches():
    # AHF_OPT_GRAPHS: captured once, replayed while the launch parameters
    # repeat, recaptured when they change; results identical to plain launches
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pops = [synth.halo_batch(seed=71, n_halos=50, n_lo=100, n_hi=100_000),
            synth.halo_batch(seed=72, n_halos=30, n_lo=100, n_hi=20_000)]
    ctx = ahf.Context(0)
    for pop in pops:
        parts = ahf.particles_from_population(pop)
        hal = ahf.halos_from_population(pop)
        prm = ahf.params_for(pop)
        ctx.set_option(ahf.OPT_GRAPHS, 0)
        ref = ctx.unbind_profile_batch(parts, hal, prm, n_bins=16, r_min_frac=0.02)
        torch.cuda.synchronize()
        ctx.set_option(ahf.OPT_GRAPHS, 1)
        out = ctx.alloc_outputs(pop.n_halos, pop.n_particles)
        prof = torch.empty((pop.n_halos, 16, 4), dtype=torch.float64, device="cuda")
        for call in range(3):
            for k in ("bound_idx", "phi", "removed_iter", "res"):
                out[k].zero_()
            prof.zero_()
            ctx.unbind_profile_batch(parts, hal, prm, n_bins=16, r_min_frac=0.02, out=out, prof=prof)
            st = ctx.stats()
            assert st["graph_launches"] == 1
            assert st["graph_captures"] == (1 if call == 0 else 0), (call, st["graph_captures"])
            torch.cuda.synchronize()
            assert torch.equal(out["res"], ref["res"])
            assert torch.equal(out["removed_iter"], ref["removed_iter"])
            assert torch.equal(prof, ref["prof"])
            res = ahf.results_to_numpy(ref["res"])
            bi, bi_r = out["bound_idx"].cpu().numpy(), ref["bound_idx"].cpu().numpy()
            for h in range(pop.n_halos):
                lo, nb = int(pop.offset[h]), int(res["n_bound"][h])
                np.testing.assert_array_equal(bi[lo:lo + nb], bi_r[lo:lo + nb])
    ctx.set_option(ahf.OPT_GRAPHS, 0)


def test_trace_fields_and_results_unchanged():
    # AHF_OPT_TRACE: monotone phase timestamps for every on-chip halo, its
    # variant and iteration count; zeros for the multi-CTA class; results
    # identical to an untraced call
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=73, n_halos=60, n_lo=100, n_hi=200_000)
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_PROMOTE, 0)               # each halo in the smallest class
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    ref = ctx.unbind_batch(parts, hal, prm)
    torch.cuda.synchronize()
    with pytest.raises(ahf.AHFError):
        ctx.trace(pop.n_halos)                      # nothing traced yet
    ctx.set_option(ahf.OPT_TRACE, 1)
    out = ctx.unbind_batch(parts, hal, prm)
    tr = ctx.trace(pop.n_halos)
    ctx.set_option(ahf.OPT_TRACE, 0)
    torch.cuda.synchronize()
    assert torch.equal(out["res"], ref["res"]) and torch.equal(out["removed_iter"], ref["removed_iter"])
    res = ahf.results_to_numpy(out["res"])
    caps = ahf.VARIANT_CAPS
    for h in range(pop.n_halos):
        n = int(pop.count[h])
        v = next((k for k, c in enumerate(caps) if n <= c), None)
        if v is None:
            assert np.all(tr[h] == 0)
            continue
        assert np.all(np.diff(tr[h, :6]) >= 0) and tr[h, 0] > 0, tr[h]
        assert tr[h, 7] & 255 == v and tr[h, 7] >> 8 == res["n_iter"][h]
    with pytest.raises(ahf.AHFError):
        ctx.trace(pop.n_halos + 1)


def test_serial_classes_same_bits():
    """AHF_OPT_SERIAL (classes one after another, each phase timed alone)
    changes nothing in the results."""
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=75, n_halos=60, n_lo=100, n_hi=100_000)
    ctx = ahf.Context(0)
    base, _, _, _ = run_gpu(pop, ctx=ctx)
    ctx.set_option(ahf.OPT_SERIAL, 1)
    ctx.set_option(ahf.OPT_TIMING, 1)
    assert ctx.get_option(ahf.OPT_SERIAL) == 1
    ser, _, _, _ = run_gpu(pop, ctx=ctx)
    st = ctx.stats()
    assert ser["res"].tobytes() == base["res"].tobytes()
    np.testing.assert_array_equal(ser["removed_iter"], base["removed_iter"])
    for h in range(pop.n_halos):          # slots past n_bound are unspecified
        lo, nb = int(pop.offset[h]), int(base["res"][h]["n_bound"])
        np.testing.assert_array_equal(ser["bound_idx"][lo:lo + nb], base["bound_idx"][lo:lo + nb])
        np.testing.assert_array_equal(ser["phi"][lo:lo + nb], base["phi"][lo:lo + nb])
    used = [k for k in range(8) if st["phase_halos"][k] > 0]
    assert used and all(st["phase_ms"][k] > 0 for k in used)
    with pytest.raises(ahf.AHFError):
        ctx.set_option(ahf.OPT_SERIAL, 2)


@pytest.mark.parametrize("case", ["single", "small_warp", "cta", "clusters"])
def test_promotion_same_bits(case):
    """AHF_OPT_PROMOTE (the default): a batch that leaves SMs idle runs in
    larger classes, with the same results as in the smallest ones."""
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = {"single": lambda: synth.single_halo(seed=synth.SEED_BASE + 1),
           "small_warp": lambda: synth.halo_batch(seed=81, n_halos=3, n_lo=150, n_hi=400),
           "cta": lambda: synth.halo_batch(seed=82, n_halos=8, n_lo=1500, n_hi=6000),
           "clusters": lambda: synth.halo_batch(seed=83, n_halos=4, n_lo=9000, n_hi=40000)}[case]()
    base, _, c0, _ = run_gpu(pop)                              # the smallest classes
    st0 = c0.stats()["phase_halos"][:8]
    ctx = ahf.Context(0)
    assert ctx.get_option(ahf.OPT_PROMOTE) == 1
    prom, _, _, _ = run_gpu(pop, ctx=ctx)
    st1 = ctx.stats()["phase_halos"][:8]
    # every halo moved up (the batches are far below the machine's capacity)
    mean0 = sum(k * n for k, n in enumerate(st0)) / max(1, sum(st0))
    mean1 = sum(k * n for k, n in enumerate(st1)) / max(1, sum(st1))
    assert sum(st1) == sum(st0) == pop.n_halos and mean1 > mean0, (st0, st1)
    assert prom["res"].tobytes() == base["res"].tobytes()
    np.testing.assert_array_equal(prom["removed_iter"], base["removed_iter"])
    for h in range(pop.n_halos):
        lo, nb = int(pop.offset[h]), int(base["res"][h]["n_bound"])
        np.testing.assert_array_equal(prom["bound_idx"][lo:lo + nb], base["bound_idx"][lo:lo + nb])
        np.testing.assert_array_equal(prom["phi"][lo:lo + nb], base["phi"][lo:lo + nb])
    with pytest.raises(ahf.AHFError):
        ctx.set_option(ahf.OPT_PROMOTE, 3)


@pytest.mark.parametrize("n_bins", [1, 7, 129, 300])
def test_profile_bin_counts(n_bins):
    # one bin, an odd count, and counts above the clusters' fused limit (128:
    # their rows then come from the standalone profile kernel); the bin
    # tables travel in the same staged copy as the halo descriptors
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=43, n_halos=40, n_lo=100, n_hi=60_000)
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    fused = ctx.unbind_profile_batch(parts, hal, prm, n_bins=n_bins, r_min_frac=0.02)
    sep = ctx.profile_batch(parts, hal, prm, fused["res"], fused["bound_idx"], n_bins=n_bins, r_min_frac=0.02)
    torch.cuda.synchronize()
    a = fused["prof"].cpu().numpy()
    b = sep.cpu().numpy()
    assert a.shape == (pop.n_halos, n_bins, 4)
    np.testing.assert_array_equal(a[:, :, 0], b[:, :, 0])
    np.testing.assert_allclose(a[:, :, 1], b[:, :, 1], rtol=1e-12, atol=0)
    np.testing.assert_allclose(a[:, :, 2:], b[:, :, 2:], rtol=1e-6, atol=0)
    res = ahf.results_to_numpy(fused["res"])
    compare(pop, prm, res, fused["bound_idx"].cpu().numpy(), fused["phi"].cpu().numpy(),
            fused["removed_iter"].cpu().numpy())
    _check_profiles(pop, prm, res, a, n_bins, 0.02)
    # the host-buffer entry stages the same tables
    hparts = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, pop.m, pop.m0, pop.coord_type)
    host = ctx.unbind_batch_host(hparts, hal, prm, n_bins=n_bins, r_min_frac=0.02)
    np.testing.assert_array_equal(host["prof"], a)

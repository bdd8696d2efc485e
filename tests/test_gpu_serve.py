"""Serving front end (ahf_serve_*): results of requests served in mixed,
continuously formed batches equal the results of unbinding each halo in an
ordinary batch (and alone); admission by ring space, ring wrap-around, and
the poll protocol's error cases."""
import time

import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu

pytestmark = pytest.mark.gpu

_FIELDS = ("n_bound", "n_member", "part_iter", "n_band", "k_vir", "n_iter", "status", "m_vir", "r_vir")


def _host_particles(pop):
    from paper_0904_3662_gb300 import ahf
    return ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, pop.m, float(pop.m0), int(pop.coord_type))


def _serve_all(srv, pop, order, deadline_s=120.0):
    """Submit the haloes in `order`, retrying on a full ring; poll until all
    have completed.  Returns {halo: (record, bound indices)}, refusals."""
    from paper_0904_3662_gb300 import ahf
    parts = _host_particles(pop)
    hal = ahf.halos_from_population(pop)
    pending, done, refused = {}, {}, 0
    todo = list(order)
    t_end = time.time() + deadline_s
    while (todo or pending) and time.time() < t_end:
        while todo:
            rid = srv.submit(parts, hal[todo[0]:todo[0] + 1])
            if rid is None:
                refused += 1
                break
            pending[rid] = todo.pop(0)
        for rid in list(pending):
            got = srv.poll(rid)
            if got is not None:
                done[pending.pop(rid)] = got
        time.sleep(0.0005)
    assert not todo and not pending, "serving did not finish in time"
    return done, refused


def _check_same(pop, done, ref):
    res = ref["res"]
    for h, (rec, bound) in done.items():
        for k in _FIELDS:
            assert rec[k] == res[k][h], (h, k, rec[k], res[k][h])
        np.testing.assert_array_equal(rec["vbulk"], res["vbulk"][h])
        lo = int(pop.offset[h])
        np.testing.assert_array_equal(bound, ref["bound_idx"][lo:lo + int(res["n_bound"][h])])


def test_served_requests_equal_batch_and_alone():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=51, n_halos=80, n_lo=100, n_hi=60_000)
    ref, prm, ctx, _ = run_gpu(pop, with_phi=False, with_removed=False)
    srv = ahf.Serve(prm, hbm_cap_bytes=1 << 30, coord_type=pop.coord_type, m0=pop.m0)
    try:
        order = list(np.random.default_rng(5).permutation(pop.n_halos))
        done, _ = _serve_all(srv, pop, order)
        _check_same(pop, done, ref)
        st = srv.stats()
        assert st["completed"] == pop.n_halos and st["submitted"] == pop.n_halos
        assert 1 <= st["batches"] <= pop.n_halos
        assert 0.0 < st["p50_us"] <= st["p99_us"]
    finally:
        srv.close()
    # and alone: three haloes of different classes, one per batch call
    for h in (int(np.argmin(pop.count)), int(np.argmax(pop.count)), pop.n_halos // 2):
        one = ahf.halos_from_population(pop)[h:h + 1]
        alone, _, _, _ = run_gpu(pop, params=prm, halos=one, ctx=ctx, with_phi=False, with_removed=False)
        for k in _FIELDS:
            assert alone["res"][k][0] == ref["res"][k][h], (h, k)


def test_ring_wraps_and_refuses_when_full():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    # ring of 262,144 slots: 64 MiB workspace allowance + 2 x 8192 records + slots x (6 floats + index)
    slots = 262_144
    cap = (64 << 20) + 2 * 8192 * 88 + slots * (6 * 4 + 8)
    pop = synth.halo_batch(seed=52, n_halos=200, n_lo=2_000, n_hi=20_000)
    assert pop.count.sum() > 3 * slots          # several passes through the ring
    ref, prm, _, _ = run_gpu(pop, with_phi=False, with_removed=False)
    srv = ahf.Serve(prm, hbm_cap_bytes=cap, coord_type=pop.coord_type, m0=pop.m0)
    try:
        done, refused = _serve_all(srv, pop, list(range(pop.n_halos)))
        _check_same(pop, done, ref)
        # refusals depend on how far submission runs ahead of the device;
        # every one of them is counted and was retried
        assert srv.stats()["rejected"] == refused
    finally:
        srv.close()


def test_masses_and_f64_coordinates_and_poll_errors():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=53, n_halos=12, n_lo=200, n_hi=9_000, coord_type=synth.COORD_F64,
                           with_masses=True)
    ref, prm, _, _ = run_gpu(pop, with_phi=False, with_removed=False)
    srv = ahf.Serve(prm, hbm_cap_bytes=1 << 30, coord_type=ahf.COORD_F64, m0=0.0)
    try:
        parts = _host_particles(pop)
        hal = ahf.halos_from_population(pop)
        # wrong mass mode / coordinate type are refused at submission
        bad = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, float(pop.m0), ahf.COORD_F64)
        with pytest.raises(ahf.AHFError) as e:
            srv.submit(bad, hal[:1])
        assert e.value.code == ahf.ERR_INVALID
        with pytest.raises(ahf.AHFError) as e:
            srv.poll(987654321)
        assert e.value.code == ahf.ERR_NOT_FOUND
        big = int(np.argmax(pop.count))
        rid = srv.submit(parts, hal[big:big + 1])
        t_end = time.time() + 60
        while time.time() < t_end:
            try:
                got = srv.poll(rid, cap=1)          # too small unless n_bound <= 1
            except ahf.AHFError as err:
                assert err.code == ahf.ERR_INVALID and "cap" in str(err)
                break
            assert got is None
            time.sleep(0.001)
        rec, bound = srv.poll(rid)                  # kept after the refused poll
        lo = int(pop.offset[big])
        np.testing.assert_array_equal(bound, ref["bound_idx"][lo:lo + int(ref["res"]["n_bound"][big])])
        with pytest.raises(ahf.AHFError) as e:
            srv.poll(rid)
        assert e.value.code == ahf.ERR_NOT_FOUND
        done, _ = _serve_all(srv, pop, list(range(pop.n_halos)))
        _check_same(pop, done, ref)
    finally:
        srv.close()

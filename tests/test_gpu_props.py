"""Integral properties (ahf_halo_properties) and catalogue matching
(ahf_match_catalogs) against the oracle, on the unbinding's own outputs."""
import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu
from tests.parity import compare, oracle_params

pytestmark = pytest.mark.gpu


def _run(pop, **kw):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop, **kw)
    out = ctx.unbind_batch(parts, hal, prm)
    props = ctx.halo_properties(parts, hal, prm, out)
    torch.cuda.synchronize()
    ctx.sync()
    host = {"res": ahf.results_to_numpy(out["res"]), "bound_idx": out["bound_idx"].cpu().numpy(),
            "phi": out["phi"].cpu().numpy(), "removed_iter": out["removed_iter"].cpu().numpy(),
            "props": props.cpu().numpy()}
    return ctx, prm, out, host


def _check_props(pop, prm, host, phi_rtol):
    compare(pop, prm, host["res"], host["bound_idx"], host["phi"], host["removed_iter"], phi_rtol=phi_rtol,
            vir_rtol=max(phi_rtol, 1e-5), exact_order=phi_rtol < 1e-9)
    op = oracle_params(prm)
    ref = O.unbind_population(pop, op, forced=host["removed_iter"], properties=True)
    checked = 0
    for h in range(pop.n_halos):
        r, o, g = host["res"][h], ref[h], host["props"][h]
        if int(r["k_vir"]) != o["k_vir"] or int(r["n_bound"]) != o["order"].shape[0]:
            continue                                  # a virial band case: different selections
        q = o["props"]
        assert g[0] == q["n"] and g[11] == (1.0 if o["k_vir"] >= 0 else 0.0)
        if q["n"] == 0:
            assert np.all(g[:11] == 0.0)
            continue
        checked += 1
        assert g[1] == pytest.approx(q["M"], rel=1e-12)
        jscale = np.abs(q["J"]).max() + 1e-12 * q["M"]
        np.testing.assert_allclose(g[2:5], q["J"], rtol=0, atol=1e-8 * jscale)
        assert g[5] == pytest.approx(q["K"], rel=1e-9)
        assert g[6] == pytest.approx(q["U"], rel=10 * phi_rtol)
        assert g[7] == pytest.approx(q["E"], rel=10 * phi_rtol * (abs(q["K"]) + abs(q["U"])) / abs(q["E"]))
        assert g[8] == pytest.approx(q["lam"], rel=10 * phi_rtol * (abs(q["K"]) + abs(q["U"])) / abs(q["E"]) + 1e-8)
        assert g[9] == pytest.approx(q["v_max"], rel=1e-9)
        assert g[10] == pytest.approx(q["r_max"], rel=1e-5)
    return checked


def test_properties_mixed_batch():
    pop = synth.halo_batch(seed=81, n_halos=60, n_lo=100, n_hi=60_000)
    _, prm, _, host = _run(pop)
    assert _check_props(pop, prm, host, 1e-5) >= 55


def test_properties_fp64_masses_and_box():
    pop = synth.halo_batch(seed=82, n_halos=20, n_lo=100, n_hi=20_000, coord_type=synth.COORD_F64,
                           with_masses=True)
    from paper_0904_3662_gb300 import ahf
    _, prm, _, host = _run(pop, precision=ahf.PREC_FP64)
    assert _check_props(pop, prm, host, 1e-11) >= 18
    tail = synth.large_tail(n_halos=2, n_lo=20_000, n_hi=40_000, n_sub=4)
    _, prm, _, host = _run(tail)
    assert _check_props(tail, prm, host, 1e-5) >= 1


def _catalogue(pop, host):
    res = host["res"]
    off = pop.offset.astype(np.int64)
    cnt = res["n_bound"].astype(np.int64)
    lists = [host["bound_idx"][off[h]:off[h] + cnt[h]] for h in range(pop.n_halos)]
    return off, cnt, lists


def test_match_catalogs_two_runs():
    torch = require_gpu()
    pop = synth.halo_batch(seed=83, n_halos=80, n_lo=100, n_hi=30_000)
    ctx, _, out_a, host_a = _run(pop)
    _, _, out_b, host_b = _run(pop, H=0.0, max_iter=1)     # another catalogue of the same particles
    off_a, cnt_a, lists_a = _catalogue(pop, host_a)
    off_b, cnt_b, lists_b = _catalogue(pop, host_b)
    # reverse the second catalogue's order: the answers must follow
    rev = np.arange(pop.n_halos)[::-1].copy()
    lists_b = [lists_b[k] for k in rev]
    off_b, cnt_b = off_b[rev].copy(), cnt_b[rev].copy()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    best, shared, xi = ctx.match_catalogs(pop.n_particles, out_a["bound_idx"], dev(off_a), dev(cnt_a),
                                          out_b["bound_idx"], dev(off_b), dev(cnt_b))
    torch.cuda.synchronize()
    ctx.sync()
    rb, rs, rx = O.match_catalogs(lists_a, lists_b)
    np.testing.assert_array_equal(best.cpu().numpy(), rb)
    np.testing.assert_array_equal(shared.cpu().numpy(), rs)
    np.testing.assert_array_equal(xi.cpu().numpy(), rx)
    ne = cnt_a > 0
    assert np.all(rb[ne] == rev[ne])                         # each halo finds itself
    # a catalogue matched with itself: xi = 1 everywhere a halo is not empty
    best, shared, xi = ctx.match_catalogs(pop.n_particles, out_a["bound_idx"], dev(off_a), dev(cnt_a),
                                          out_a["bound_idx"], dev(off_a), dev(cnt_a))
    torch.cuda.synchronize()
    assert np.all(best.cpu().numpy()[ne] == np.arange(pop.n_halos)[ne]) and np.all(xi.cpu().numpy()[ne] == 1.0)


def test_match_catalogs_reports_bad_input():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    ctx = ahf.Context(0)

    def dev(a):
        return torch.tensor(a, dtype=torch.int64, device="cuda")
    ids = dev([0, 1, 2, 3, 2])                               # id 2 in both haloes of the second
    best, shared, xi = ctx.match_catalogs(10, ids, dev([0]), dev([3]), ids, dev([0, 3]), dev([3, 2]))
    torch.cuda.synchronize()
    with pytest.raises(ahf.AHFError) as e:
        ctx.sync()
    assert "two haloes" in str(e.value)
    best, shared, xi = ctx.match_catalogs(3, ids, dev([0]), dev([4]), ids, dev([0]), dev([2]))
    torch.cuda.synchronize()
    with pytest.raises(ahf.AHFError) as e:
        ctx.sync()
    assert "out of range" in str(e.value)

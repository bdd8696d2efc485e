"""Comparison of the CUDA path's outputs with the CPU oracle.

Tolerances (floating point, from the method's stated accuracy target):
  * phi, M_vir, R_vir: relative error <= 1e-5;
  * bound sets identical as sets, listed in radial order (the GPU orders by
    its float32 radius, so particles whose radii agree to float32 resolution
    may appear in either order; phi is compared particle by particle).
    Particles whose escape margin
    |(|u|^2 - 2|phi|) / 2|phi|| lies below `band` (1e-5) may be decided either
    way; the oracle then replays the GPU's decision for exactly those
    particles (and only those) so that later iterations stay comparable.
  * the virial crossing index may differ only when the oracle's own
    crossing test at the GPU's index is within 1e-5 of equality.
Integer outputs (removal iteration per candidate, iteration counts, member
counts, bound lists) must match exactly after the replay.
"""
import math

import numpy as np

from oracle import ahf_oracle as O

PHI_RTOL = 1e-5
VIR_RTOL = 1e-5


def fp64_rtol(pop):
    """Relative tolerance of phi, M_vir and R_vir for the all-FP64 mode.  The
    GPU's sums there are exact (128-bit fixed point) and rounded once; the
    oracle's are sequential FP64 sums (np.cumsum), whose relative error is at
    most (n - 1) u for n positive terms (u = 2^-53; recursive summation).
    With n the largest candidate count, twice that bound plus a few roundings
    of the final combination."""
    n = float(np.max(pop.count)) if len(pop.count) else 1.0
    return 2.0 * n * 2.0 ** -53 + 1e-14
# The mixed-precision kernels sort by r = sqrt(fma(dz, dz, fma(dy, dy, dx dx)))
# in float, each offset d the correctly rounded float of the exact offset.
# With u = 2^-24: the offsets add at most 2u to r^2, the three roundings of
# the sum 3u, so r^2 is within 5u and r within 2.5u + u (the sqrt's own
# rounding) = 3.5u of the exact radius.  Two particles whose exact radii
# differ by less than 7u relative may therefore come out in either order.
RADIUS_RTOL = 7.0 * 2.0 ** -24


def _positions(ref_idx, idx):
    """Position in ref_idx of every entry of idx (both permutations of one set)."""
    order = np.argsort(ref_idx, kind="stable")
    return order[np.searchsorted(ref_idx, idx, sorter=order)]


def oracle_params(p):
    return O.Params(G=p.G, H=p.H, delta_rho=p.delta_rho, r_soft=p.r_soft, box=p.box,
                    max_iter=p.max_iter, band=p.band, vbulk_initial=bool(p.variant & 1),
                    retruncate=bool(p.variant & 2), rise_edge=bool(p.variant & 4))


def compare(pop, params, res, bound_idx, phi, removed_iter, halos=None, member_idx=None,
            check_phi=True, phi_rtol=PHI_RTOL, vir_rtol=VIR_RTOL, exact_order=False, parent=None):
    """res: numpy RESULT_DTYPE array; bound_idx/phi/removed_iter: host numpy
    arrays over the candidate slots; parent: compare with the hierarchical
    unbinding of that forest.  Returns summary statistics; raises
    AssertionError on a mismatch."""
    hs = range(pop.n_halos) if halos is None else halos
    op = oracle_params(params)
    if parent is None:
        ref = O.unbind_population(pop, op, halos=hs, member_idx=member_idx, forced=removed_iter)
    else:
        ref = O.unbind_hierarchy(pop, op, parent, member_idx=member_idx, forced=removed_iter)
    worst_phi = 0.0
    worst_vir = 0.0
    worst_order = 0.0
    n_band = 0
    for h in hs:
        o = ref[h]
        r = res[h]
        lo = int(pop.offset[h])
        n = int(pop.count[h])
        msg = f"halo {h} (count {n})"
        np.testing.assert_array_equal(removed_iter[lo:lo + n], o["removed_iter"], err_msg=msg)
        assert int(r["n_member"]) == o["n_member"], msg
        assert int(r["n_iter"]) == o["n_iter"], (msg, int(r["n_iter"]), o["n_iter"])
        assert int(r["part_iter"]) == o["part_iter"], msg
        nb = int(r["n_bound"])
        assert nb == o["order"].shape[0], (msg, nb, o["order"].shape[0])
        gb = bound_idx[lo:lo + nb]
        # the bound set is unique: identical as a set
        np.testing.assert_array_equal(np.sort(gb), np.sort(o["bound_idx"]), err_msg=msg)
        # the order is radial: the GPU sorts by its float32 radius, so
        # particles whose radii agree to float32 resolution may swap
        if exact_order:
            # FP64 radii equal the oracle's: the order is the oracle's exactly
            np.testing.assert_array_equal(gb, o["bound_idx"], err_msg=msg)
        pos = _positions(o["bound_idx"], gb)
        r_o = o["r"][pos]
        if nb > 1:
            a, b = r_o[:-1], r_o[1:]
            pos_a = a > 0.0
            inv = float(np.max((a[pos_a] - b[pos_a]) / a[pos_a], initial=0.0))
            worst_order = max(worst_order, inv)
            assert inv <= RADIUS_RTOL, (msg, "bound list not in radial order", inv / 2.0 ** -24)
        st = int(r["status"])
        n_band += int(r["n_band"])
        if nb and check_phi:
            ph = phi[lo:lo + nb].astype(np.float64)
            rel = np.abs(ph / o["phi"][pos] - 1.0)
            worst_phi = max(worst_phi, float(rel.max()))
            assert rel.max() <= phi_rtol, (msg, float(rel.max()))
        # virial crossing
        if st != o["status"] or abs(int(r["k_vir"]) - o["k_vir"]) > 0:
            _virial_band_ok(o, r, op, msg)
        else:
            if o["m_vir"] > 0:
                e1 = abs(r["m_vir"] / o["m_vir"] - 1.0)
                e2 = abs(r["r_vir"] / o["r_vir"] - 1.0)
                worst_vir = max(worst_vir, e1, e2)
                assert e1 <= vir_rtol and e2 <= vir_rtol, (msg, e1, e2)
            else:
                assert r["m_vir"] == 0.0 and r["r_vir"] == 0.0, msg
        if nb:
            err = np.abs(r["vbulk"] - o["vbulk"])
            tol = vbulk_tolerance(pop, h, o, fp64=getattr(params, "precision", 0) == 1, rtol=vir_rtol,
                                  member_idx=member_idx)
            assert np.all(err <= tol), (msg, r["vbulk"], o["vbulk"], tol)
    return {"worst_phi_rel": worst_phi, "worst_vir_rel": worst_vir, "n_band": n_band,
            "worst_order_inversion": worst_order,
            "halos": len(list(hs))}


def vbulk_tolerance(pop, h, o, fp64, rtol, member_idx=None):
    """Per-component bound on |v_bulk(GPU) - v_bulk(oracle)|.

    v_bulk = sum m v / sum m over the bound set.  The GPU forms every product
    m v once in its working precision (float in the mixed mode, where a
    float64 input velocity or mass is also rounded to float once; double in
    the FP64 mode) and sums the rounded products exactly in 64-bit fixed
    point.  Each product is turned into fixed point with an error of at most
    half the quantum 2^-s, where the scale s = 61 - ceil(log2 n) - e (n the
    members, 2^e <= the largest |m v| among the halo's members) gives
    2^-s < 2 n max|m v| 2^-61.  So the error of the sum is at most
    eps sum |m v| + n_bound n max|m v| 2^-61 (eps = 2^-22 for float: two
    roundings of 2^-24 with margin; 2^-51 for double), divided by sum m.
    A relative rtol of |v_bulk| is allowed on top (the stated accuracy)."""
    lo, n = int(pop.offset[h]), int(pop.count[h])
    cand = np.arange(lo, lo + n) if member_idx is None else np.asarray(member_idx[lo:lo + n], np.int64)
    mc = np.full(n, float(pop.m0)) if pop.m is None else np.asarray(pop.m[cand], np.float64)
    vc = np.stack([np.asarray(a[cand], np.float64) for a in (pop.vx, pop.vy, pop.vz)], axis=1)
    mv_max = np.abs(mc[:, None] * vc).max(axis=0)
    bi = o["bound_idx"]
    mb = np.asarray(o["m"], np.float64)
    vb = np.stack([np.asarray(a[bi], np.float64) for a in (pop.vx, pop.vy, pop.vz)], axis=1)
    mv_abs = np.abs(mb[:, None] * vb).sum(axis=0)
    eps = 2.0 ** -51 if fp64 else 2.0 ** -22
    n_m = float(o["n_member"])
    floor = (eps * mv_abs + float(bi.shape[0]) * n_m * mv_max * 2.0 ** -61) / float(mb.sum())
    return rtol * np.abs(o["vbulk"]) + floor


def _virial_band_ok(o, r, op, msg):
    """A differing crossing index is acceptable only if the oracle's test at
    the GPU's index is within 1e-5 of equality (both choices are valid)."""
    k = int(r["k_vir"])
    rs = o["r"]
    if rs.shape[0] == 0:
        raise AssertionError((msg, "status differs on an empty set"))
    mk = np.cumsum(o["m"])
    crit = op.delta_rho * 4.0 * math.pi / 3.0
    ks = [k, o["k_vir"]]
    for kk in ks:
        if 0 <= kk < rs.shape[0] - 1:
            lhs, rhs = mk[kk], crit * rs[kk + 1] ** 3
            if abs(lhs / rhs - 1.0) < VIR_RTOL:
                return
    raise AssertionError((msg, "virial crossing differs outside the band", k, o["k_vir"], int(r["status"]),
                          o["status"]))


def check_profiles(pop, prm, res, prof, n_bins, f, halos=None):
    """Profile rows against the oracle's: counts may move between
    neighbouring bins only for particles within 2e-5 of an edge; masses
    accordingly; shell density and v_circ to 1e-5 where no particle is on an
    edge."""
    hs = range(pop.n_halos) if halos is None else halos
    ref = O.unbind_population(pop, oracle_params(prm), halos=hs, forced=None, n_bins=n_bins, r_min_frac=f)
    for h in hs:
        o = ref[h]
        gp = prof[h]
        if o["order"].shape[0] == 0:
            assert np.all(gp == 0.0)
            continue
        r_out = float(res[h]["r_vir"]) if res[h]["r_vir"] > 0 else float(o["r"][-1])
        edges = r_out * f ** (1.0 - np.arange(n_bins + 1) / n_bins)
        edges[-1] = r_out
        near = np.zeros(n_bins, dtype=np.int64)
        for b in range(n_bins):
            for e in (edges[b], edges[b + 1]):
                near[b] += int(np.sum(np.abs(o["r"] / e - 1.0) < 2e-5))
        # counts may move between neighbouring bins only for particles on an edge
        assert np.all(np.abs(gp[:, 0] - o["profile"][:, 0]) <= near), (h, gp[:, 0], o["profile"][:, 0])
        mp = float(o["m"].max())
        cum_near = np.cumsum(near)
        assert np.all(np.abs(gp[:, 1] - o["profile"][:, 1]) <= cum_near * mp + 1e-9 * o["profile"][:, 1] + 1e-6)
        ok = near == 0
        np.testing.assert_allclose(gp[ok, 2], o["profile"][ok, 2], rtol=1e-5)
        np.testing.assert_allclose(gp[ok, 3], o["profile"][ok, 3], rtol=1e-5)

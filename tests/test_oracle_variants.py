"""Pins of the oracle's method variants: the bulk velocity fixed from the
initial set, the second unbinding pass within r_vir (Appendix A's
truncation at r_vir), the subhalo edge at the rise of the density profile,
gas thermal energy and the host/subhalo hierarchy."""
import dataclasses

import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import synth


def _unbind(d, v, m, **kw):
    prm = O.Params(H=0.0, **kw)
    return O.unbind_halo(np.asarray(d, float), np.asarray(v, float), np.asarray(m, float),
                         np.ones(len(m), dtype=bool), prm)


def test_initial_bulk_velocity_keeps_a_comoving_particle():
    # A: 1e12 at r = 1, at rest; B: 2e11 at r = 50 moving +3000 km/s; C: 1e9 at
    # r = 100 moving +600 km/s.  Iteration 1 (both readings): v_bulk =
    # 2e11 * 3000 / 1.201e12 = 499.6; B: |u| = 2500 > v_esc(B) = 454 -> removed;
    # C: |u| = 100 < v_esc(C) = sqrt(2 G 1.201e12 / 100) = 321 -> kept.
    # Iteration 2: the current set's v_bulk is 600 * 1e9 / 1.001e12 = 0.6, so
    # C has |u| = 599 > v_esc(C) = sqrt(2 G 1.001e12 / 100) = 293 -> removed;
    # with the initial set's v_bulk (499.6) C keeps |u| = 100 -> bound.
    d = [[1.0, 0, 0], [50.0, 0, 0], [100.0, 0, 0]]
    v = [[0.0, 0, 0], [3000.0, 0, 0], [600.0, 0, 0]]
    m = [1e12, 2e11, 1e9]
    o = _unbind(d, v, m)
    assert o["removed_iter"].tolist() == [0, 1, 2] and o["order"].tolist() == [0]
    o = _unbind(d, v, m, vbulk_initial=True)
    assert o["removed_iter"].tolist() == [0, 1, 0] and o["order"].tolist() == [0, 2]
    # without the fast particle the readings agree
    o1 = _unbind(d[::2], v[::2], m[::2])
    o2 = _unbind(d[::2], v[::2], m[::2], vbulk_initial=True)
    assert o1["removed_iter"].tolist() == o2["removed_iter"].tolist()


def _halo(seed):
    pop = synth.halo_batch(seed=seed, n_halos=6, n_lo=300, n_hi=20_000)
    return pop


def test_retruncation_is_a_second_pass_within_r_vir():
    pop = _halo(91)
    base = O.Params()
    one = O.unbind_population(pop, base)
    two = O.unbind_population(pop, dataclasses.replace(base, retruncate=True))
    for h in range(pop.n_halos):
        a, b = one[h], two[h]
        # the second pass keeps a subset of the first pass's bound set inside r_vir
        inside = set(a["bound_idx"][a["r"] <= a["r_vir"]].tolist()) if a["r_vir"] > 0 else set(a["bound_idx"].tolist())
        assert set(b["bound_idx"].tolist()) <= inside
        assert b["n_member"] == len(inside)
        # removal iterations are the first pass's
        np.testing.assert_array_equal(b["removed_iter"], a["removed_iter"])
        # and the second pass is the plain unbinding of exactly those candidates
        pidx, d, v, m, _ = O.gather_sphere(pop, h)
        sel = np.isin(pidx, sorted(inside))
        c = O.unbind_halo(d, v, m, sel, base)
        np.testing.assert_array_equal(np.sort(pidx[c["order"]]), np.sort(b["bound_idx"]))
        assert c["n_iter"] == b["n_iter"] and c["r_vir"] == b["r_vir"]


def test_retruncation_of_a_halo_inside_its_r_vir_changes_nothing():
    # a cold uniform sphere whose mean density stays above delta_rho to its
    # edge (r_vir beyond the outermost particle): the second pass sees the
    # same set and gives the same result
    rng = np.random.default_rng(3)
    n, R = 2000, 50.0
    d = rng.normal(size=(n, 3))
    d *= (R * rng.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    m = np.full(n, 1e9)
    v = np.zeros((n, 3))
    prm = O.Params(H=0.0)
    a = O.unbind_halo(d, v, m, np.ones(n, bool), prm)
    assert a["status"] & O.RVIR_BEYOND_EDGE and a["r_vir"] >= a["r"][-1]
    b = O.retruncate_halo(a, d, v, m, prm)
    np.testing.assert_array_equal(b["order"], a["order"])
    np.testing.assert_array_equal(b["phi"], a["phi"])
    assert b["r_vir"] == a["r_vir"] and b["n_iter"] == 1


def test_retruncation_unbinds_what_the_outer_mass_held():
    # a core of 400 particles (r < 20) plus a massive shell at r = 400 far
    # beyond r_vir; one test particle at r = 30 moving just below the escape
    # speed of the whole set: bound in the first pass (the shell adds
    # G m_shell / 400 to |phi|), outside the shell's help in the second pass
    rng = np.random.default_rng(4)
    core = rng.normal(size=(400, 3))
    core *= (20.0 * rng.uniform(0, 1, 400) ** (1 / 3) / np.linalg.norm(core, axis=1))[:, None]
    shell = rng.normal(size=(200, 3))
    shell *= (400.0 / np.linalg.norm(shell, axis=1))[:, None]
    t = np.array([[30.0, 0.0, 0.0]])
    d = np.concatenate([core, t, shell])
    m = np.concatenate([np.full(400, 1e9), [1e6], np.full(200, 2e9)])
    prm = O.Params(H=0.0)
    G = prm.G
    phi_all = -G * (400 * 1e9 / 30.0 + 200 * 2e9 / 400.0)       # the test particle's phi, all present
    phi_core = -G * (400 * 1e9 / 30.0)                          # without the shell
    speed = 0.5 * (np.sqrt(2 * abs(phi_all)) + np.sqrt(2 * abs(phi_core)))
    v = np.zeros_like(d)
    v[400, 0] = speed
    a = O.unbind_halo(d, v, m, np.ones(len(m), bool), prm)
    assert 400 in a["order"].tolist()                            # bound with the shell
    assert a["r_vir"] < 400.0                                    # the shell is outside r_vir
    b = O.retruncate_halo(a, d, v, m, prm)
    assert 400 not in b["order"].tolist()                        # unbound without it
    assert set(b["order"].tolist()) == set(range(400))


def test_gas_thermal_energy_in_the_escape_test():
    # a particle of negligible mass at r = 30 around a 1e12 point-like core,
    # |v| = 0.9 v_esc: bound as collisionless matter; with a thermal energy
    # u_th = 0.2 v_esc^2 the test |v|^2 + 2 u_th = 0.81 + 0.4 > 1 removes it;
    # with u_th = 0.05 v_esc^2 (0.81 + 0.1 < 1) it stays
    prm = O.Params(H=0.0)
    d = np.array([[0.5, 0, 0], [30.0, 0, 0]])
    m = np.array([1e12, 1.0])
    v_esc2 = 2 * prm.G * (1e12 + 1.0) / 30.0
    v = np.array([[0.0, 0, 0], [0.9 * np.sqrt(v_esc2), 0, 0]])
    ins = np.ones(2, bool)
    assert O.unbind_halo(d, v, m, ins, prm)["removed_iter"].tolist() == [0, 0]
    hot = O.unbind_halo(d, v, m, ins, prm, u_th=np.array([0.0, 0.2 * v_esc2]))
    assert hot["removed_iter"].tolist() == [0, 1]
    warm = O.unbind_halo(d, v, m, ins, prm, u_th=np.array([0.0, 0.05 * v_esc2]))
    assert warm["removed_iter"].tolist() == [0, 0]
    # no gas (u_th = 0 everywhere) is the collisionless unbinding, bit for bit
    pop = _halo(95)
    for h in range(pop.n_halos):
        pidx, dd, vv, mm, inside = O.gather_sphere(pop, h)
        a = O.unbind_halo(dd, vv, mm, inside, prm)
        b = O.unbind_halo(dd, vv, mm, inside, prm, u_th=np.zeros(len(mm)))
        np.testing.assert_array_equal(a["removed_iter"], b["removed_iter"])
        np.testing.assert_array_equal(a["phi"], b["phi"])
    # a gas cloud hot enough everywhere is empty
    rng = np.random.default_rng(8)
    dd = rng.normal(0, 20, (500, 3))
    mm = np.full(500, 1e8)
    hotcloud = O.unbind_halo(dd, np.zeros_like(dd), mm, np.ones(500, bool), prm, u_th=np.full(500, 1e7))
    assert hotcloud["status"] & O.EMPTY and hotcloud["n_iter"] == 1


def _host_with_subhaloes(seed=5):
    """A host NFW halo with three subhaloes (one holding a sub-subhalo), as a
    population whose haloes share particles through member lists: slots are
    distinct, particles are not.  Returns (pop, member_idx, parent)."""
    rng = np.random.default_rng(seed)
    parts_p, parts_v = [], []
    p, v = synth.sample_nfw(rng, 20000, 10.0, 200.0)
    parts_p.append(p)
    parts_v.append(v)
    subs = [((80.0, 0.0, 0.0), (150.0, 0.0, 0.0), 800), ((0.0, 110.0, 0.0), (0.0, -120.0, 40.0), 600),
            ((-70.0, -70.0, 0.0), (60.0, 60.0, 0.0), 500)]
    centres = [(0.0, 0.0, 0.0)]
    for c, vb, n in subs:
        p, v = synth.sample_nfw(rng, n, 12.0, 25.0, trunc=1.0)
        parts_p.append(p + np.array(c))
        parts_v.append(v + np.array(vb))
        centres.append(c)
    # a sub-subhalo inside the second subhalo
    c2 = (5.0, 112.0, 3.0)
    p, v = synth.sample_nfw(rng, 150, 12.0, 8.0, trunc=1.0)
    parts_p.append(p + np.array(c2))
    parts_v.append(v + np.array(subs[1][1]) + np.array([0.0, 0.0, 30.0]))
    centres.append(c2)
    pos = np.concatenate(parts_p)
    vel = np.concatenate(parts_v)
    n = pos.shape[0]
    radii = [400.0, 40.0, 55.0, 49.0, 10.0]
    parent = [-1, 0, 0, 0, 2]
    members, offsets, counts = [], [], []
    for c, R in zip(centres, radii):
        d = pos - np.array(c)
        sel = np.nonzero((d * d).sum(axis=1) <= (1.2 * R) ** 2)[0]
        offsets.append(sum(counts))
        counts.append(len(sel))
        members.append(sel)
    member_idx = np.concatenate(members).astype(np.int64)
    f = np.float32
    pop = synth.Population(name="host_with_subhaloes", coord_type=synth.COORD_F32_REL,
                           x=pos[:, 0].astype(f), y=pos[:, 1].astype(f), z=pos[:, 2].astype(f),
                           vx=vel[:, 0].astype(f), vy=vel[:, 1].astype(f), vz=vel[:, 2].astype(f),
                           m=None, m0=synth.PARTICLE_MASS, box=0.0, centre=np.array(centres),
                           radius=np.array(radii), offset=np.array(offsets, np.int64),
                           count=np.array(counts, np.int64), r200=np.zeros(5), conc=np.zeros(5))
    return pop, member_idx, np.array(parent)


def test_hierarchy_depths_and_forest_checks():
    assert O.halo_depths([-1, 0, 1, -1, 3, 0]).tolist() == [0, 1, 2, 0, 1, 1]
    for bad in ([1, 0], [0], [-1, 5], [-2]):
        try:
            O.halo_depths(bad)
        except ValueError:
            continue
        raise AssertionError(bad)


def test_hierarchy_excludes_what_subhaloes_bound():
    pop, mi, parent = _host_with_subhaloes()
    prm = O.Params()
    hier = O.unbind_hierarchy(pop, prm, parent, member_idx=mi)
    flat = O.unbind_population(pop, prm, member_idx=mi)
    # the deepest haloes are unbound exactly as on their own
    for h in (1, 3, 4):
        np.testing.assert_array_equal(hier[h]["bound_idx"], flat[h]["bound_idx"])
    # a subhalo with a sub-subhalo loses that one's bound particles
    sub_sub = set(hier[4]["bound_idx"].tolist())
    assert sub_sub and not sub_sub & set(hier[2]["bound_idx"].tolist())
    # the host keeps none of its descendants' bound particles, but can bind
    # what a subhalo removed
    taken = set()
    for h in (1, 2, 3, 4):
        taken |= set(hier[h]["bound_idx"].tolist())
    host = set(hier[0]["bound_idx"].tolist())
    assert not host & taken
    removed_by_subs = set()
    for h in (1, 2, 3):
        lo, n = int(pop.offset[h]), int(pop.count[h])
        ri = hier[h]["removed_iter"]
        removed_by_subs |= set(mi[lo:lo + n][ri > 0].tolist())
    assert host & removed_by_subs
    # excluded candidates count as outside the host's sphere
    lo, n = int(pop.offset[0]), int(pop.count[0])
    excluded = np.isin(mi[lo:lo + n], sorted(taken))
    assert np.all(hier[0]["removed_iter"][excluded] == -1)
    assert hier[0]["n_member"] == flat[0]["n_member"] - int(excluded.sum())
    # without parents the hierarchy is the flat unbinding
    none = O.unbind_hierarchy(pop, prm, np.full(5, -1), member_idx=mi)
    for h in range(5):
        np.testing.assert_array_equal(none[h]["bound_idx"], flat[h]["bound_idx"])


def test_rise_edge_truncates_at_the_density_minimum():
    # Sect. 2.1: a subhalo whose overdensity never drops below the threshold
    # ends where its density profile rises.  The designed haloes (16 shells
    # of n particles, density halving per shell to shell 11, then growing)
    # end with the last particle of shell 11; the mean density at the edge
    # is still far above delta_rho (no virial crossing inside the set).
    pop = synth.shell_profile_batch(rise=True)
    base = O.unbind_population(pop, O.Params())
    rise = O.unbind_population(pop, O.Params(rise_edge=True))
    for h in range(pop.n_halos):
        n = int(pop.count[h]) // 16
        a, b = base[h], rise[h]
        assert a["status"] == O.RVIR_BEYOND_EDGE and b["status"] == O.RVIR_BEYOND_EDGE | O.RISE_EDGE
        assert a["order"].shape[0] == pop.count[h]                   # all bound, as designed
        k = 12 * n - 1
        assert b["k_vir"] == k
        assert b["r_vir"] == b["r"][k] and b["m_vir"] == pytest.approx(pop.m0 * (k + 1), rel=1e-12)
        # the minimum found independently: shell densities from the designed
        # counts and the particles' radii, by histogram over the shell edges
        r = np.sort(b["r"])
        edges = np.concatenate([[0.0], r[n - 1::n]])
        cnt, _ = np.histogram(r, bins=edges)
        rho = cnt * pop.m0 / (4.0 / 3.0 * np.pi * np.diff(edges ** 3))
        assert int(np.argmin(rho[8:])) + 8 == 11 and rho[12] > rho[11] < rho[10]
        # the rest of the result is the method's
        for f in ("removed_iter", "order", "phi"):
            np.testing.assert_array_equal(a[f], b[f])


def test_rise_edge_leaves_other_haloes_alone():
    # a falling profile has no rise; a halo with a virial crossing keeps it;
    # fewer than 64 members never take the variant
    fall = synth.shell_profile_batch(rise=False)
    a = O.unbind_population(fall, O.Params())
    b = O.unbind_population(fall, O.Params(rise_edge=True))
    for h in range(fall.n_halos):
        assert a[h]["status"] == b[h]["status"] == O.RVIR_BEYOND_EDGE
        assert (a[h]["k_vir"], a[h]["r_vir"], a[h]["m_vir"]) == (b[h]["k_vir"], b[h]["r_vir"], b[h]["m_vir"])
    pop = synth.halo_batch(seed=95, n_halos=10, n_lo=300, n_hi=20_000)
    a = O.unbind_population(pop, O.Params())
    b = O.unbind_population(pop, O.Params(rise_edge=True))
    for h in range(pop.n_halos):
        if not a[h]["status"] & O.RVIR_BEYOND_EDGE:
            assert (a[h]["k_vir"], a[h]["r_vir"], a[h]["status"]) == (b[h]["k_vir"], b[h]["r_vir"], b[h]["status"])
    r = np.linspace(1.0, 2.0, 63)
    assert O.rise_edge(r, np.ones(63)) is None


def test_rise_edge_uses_shell_masses():
    # a shallow minimum: relative shell densities ... 1.08, 1.00, 1.05 ... at
    # shells 9, 10, 11; the edge is the end of shell 10 (the enclosed mass
    # over a shell's volume would put it at shell 9)
    rel = [2.0 ** (9 - s) * 1.08 for s in range(9)] + [1.08, 1.0, 1.05, 1.2, 1.4, 1.6, 1.8]
    pop = synth.shell_profile_batch(seed=77, n_shells=(400,), rho_shells=rel, sigma_v=0.0)
    o = O.unbind_population(pop, O.Params(rise_edge=True))[0]
    assert o["status"] & O.RISE_EDGE and o["k_vir"] == 11 * 400 - 1

"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to brute force, to Appendix A's
integral evaluated literally, to an analytic potential, to an invariant the
method must satisfy, or to a hand-worked case.  Planted mistakes (see
test_oracle_planted.py) show that the plausible slips fail at least one pin.
"""
import copy
import math

import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import synth

G = synth.G_GRAV


# --- phi: brute force ------------------------------------------------------

def _sorted(rng, n, ties=False, zero=False):
    r = rng.uniform(0.01, 100.0, n)
    if ties:
        r[: n // 4] = r[n // 4: n // 2]          # duplicate radii
    if zero:
        r[0] = 0.0
    m = rng.uniform(0.5, 2.0, n) * 1e8
    o = np.lexsort((np.arange(n), r))
    return r[o], m[o]


@pytest.mark.parametrize("n,ties,zero", [(1, False, False), (2, False, False), (17, True, False),
                                         (500, True, True), (2000, False, False)])
def test_phi_matches_bruteforce(n, ties, zero):
    rng = np.random.default_rng(n)
    r, m = _sorted(rng, n, ties, zero)
    a = O.potential_sorted(r, m, G)
    b = O.potential_bruteforce(r, m, G)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_phi_softened_matches_bruteforce():
    rng = np.random.default_rng(7)
    r, m = _sorted(rng, 300, ties=True, zero=True)
    a = O.potential_sorted(r, m, G, r_soft=5.0)
    b = O.potential_bruteforce(r, m, G, r_soft=5.0)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_phi_hand_worked():
    # G = 1, unit masses at r = 1, 2, 4:
    #   phi_1 = -(1/1 + 1/2 + 1/4)          = -1.75
    #   phi_2 = -(1/2 [inner] + 1/2 + 1/4)  = -1.25
    #   phi_3 = -(2/4 [inner] + 1/4)        = -0.75
    phi = O.potential_sorted(np.array([1.0, 2.0, 4.0]), np.ones(3), 1.0)
    np.testing.assert_allclose(phi, [-1.75, -1.25, -0.75], rtol=1e-15)
    # a particle at r = 0 keeps the other particles' outer terms only
    phi = O.potential_sorted(np.array([0.0, 2.0]), np.array([3.0, 1.0]), 1.0)
    np.testing.assert_allclose(phi, [-0.5, -2.0], rtol=1e-15)


# --- phi: Appendix A's integral evaluated literally --------------------------

def _phi_appendix_a(r, m, Gc):
    """phi(r_i) = G int_0^{r_i} M(<r')/r'^2 dr' + phi_0,
    phi_0 = -(G int_0^{r_t} M(<r')/r'^2 dr' + G M_t / r_t), r_t = outermost radius.
    M(<r') is the step function of the sorted list; each piece integrates
    exactly as M * (1/a - 1/b) on (a, b)."""
    n = len(r)
    integral = np.zeros(n)
    acc = 0.0
    for i in range(1, n):
        m_enc = float(np.sum(m[:i]))                # M(<r') on (r_{i-1}, r_i)
        if r[i] > r[i - 1]:
            acc += m_enc * (1.0 / r[i - 1] - 1.0 / r[i])
        integral[i] = acc
    r_t = r[-1]
    m_t = float(np.sum(m))
    phi0 = -(Gc * integral[-1] + Gc * m_t / r_t)
    return Gc * integral + phi0


def test_phi_matches_appendix_a_integral():
    rng = np.random.default_rng(11)
    r, m = _sorted(rng, 400)
    np.testing.assert_allclose(O.potential_sorted(r, m, G), _phi_appendix_a(r, m, G), rtol=1e-10)


# --- phi: analytic profiles ----------------------------------------------------

def test_phi_uniform_sphere_analytic():
    rng = np.random.default_rng(3)
    n, R, mp = 1_000_000, 100.0, 1e6
    r = np.sort(R * rng.uniform(0, 1, n) ** (1 / 3))
    m = np.full(n, mp)
    phi = O.potential_sorted(r, m, G)
    M = n * mp
    exact = -G * M * (3 * R * R - r * r) / (2 * R ** 3)
    rel = np.abs(phi / exact - 1.0)
    sel = r > 5.0                      # Poisson noise dominates the innermost few
    assert np.median(rel[sel]) < 2e-3
    assert rel[sel].max() < 2e-2


def test_phi_truncated_nfw_analytic():
    rng = np.random.default_rng(5)
    c, r200 = 10.0, 160.0
    pos, _ = synth.sample_nfw(rng, 400_000, c, r200)
    r = np.sort(np.sqrt((pos ** 2).sum(axis=1)))
    mp = 1e7
    phi = O.potential_sorted(r, np.full(r.shape[0], mp), G)
    rs, rt = r200 / c, 2 * r200
    ms = r.shape[0] * mp / float(synth.m_nfw(rt / rs))          # 4 pi rho_s r_s^3
    exact = -G * ms * (np.log1p(r / rs) / r - 1.0 / (rs + rt))
    rel = np.abs(phi / exact - 1.0)
    sel = r > 0.05 * rs
    assert np.median(rel[sel]) < 3e-3
    assert rel[sel].max() < 3e-2


def test_phi_monotone_and_outer_value():
    rng = np.random.default_rng(9)
    r, m = _sorted(rng, 3000)
    phi = O.potential_sorted(r, m, G)
    assert np.all(np.diff(phi) >= -1e-12 * np.abs(phi[:-1]))
    assert phi[-1] == pytest.approx(-G * m.sum() / r[-1], rel=1e-13)


# --- virial radius ---------------------------------------------------------------

def test_virial_identity_and_counting():
    pop = synth.single_halo()
    res = O.unbind_population(pop, O.Params())[0]
    p = O.Params()
    r_vir, m_vir = res["r_vir"], res["m_vir"]
    assert m_vir / (4.0 / 3.0 * math.pi * r_vir ** 3) == pytest.approx(p.delta_rho, rel=1e-12)
    # brute-force count of the final set inside r_vir (equal masses)
    n_in = int(np.sum(res["r"] <= r_vir))
    assert n_in * pop.m0 == pytest.approx(m_vir, rel=1e-12)
    # the next particle lies beyond r_vir, the last inside lies within it
    k = res["k_vir"]
    assert res["r"][k] <= r_vir < res["r"][k + 1]
    # M_vir close to the generator's M_200 (sampling noise and unbinding)
    assert abs(r_vir / pop.r200[0] - 1.0) < 0.05


def test_virial_uniform_sphere_closed_form():
    # Uniform sphere of mass M, radius R: mean density inside r <= R is
    # 3M/(4 pi R^3); choose delta_rho below it so r_vir = R_edge exactly
    # cannot cross inside -> beyond-edge flag and r_vir = (3M/(4 pi drho))^(1/3).
    rng = np.random.default_rng(1)
    n, R, mp = 20_000, 10.0, 1.0
    r = np.sort(R * rng.uniform(0, 1, n) ** (1 / 3))
    m = np.full(n, mp)
    drho = 0.5 * 3 * n * mp / (4 * math.pi * R ** 3)
    r_vir, m_vir, k, st = O.virial(r, m, drho)
    assert st & O.RVIR_BEYOND_EDGE
    assert r_vir == pytest.approx((3 * n * mp / (4 * math.pi * drho)) ** (1 / 3), rel=1e-14)
    assert r_vir == pytest.approx(R * 2 ** (1 / 3), rel=1e-12)


def test_virial_none_for_diffuse_set():
    r = np.array([100.0, 200.0])
    m = np.array([1.0, 1.0])
    r_vir, m_vir, k, st = O.virial(r, m, 1.0)
    assert st & O.RVIR_NONE and r_vir == 0.0 and m_vir == 0.0


# --- the unbinding loop ----------------------------------------------------------

def _single(pop):
    return O.gather_sphere(pop, 0)


def test_idempotent():
    pop = synth.single_halo()
    p = O.Params()
    pidx, d, v, m, inside = _single(pop)
    a = O.unbind_halo(d, v, m, inside, p)
    keep = np.zeros_like(inside)
    keep[a["order"]] = True
    b = O.unbind_halo(d, v, m, keep, p)
    assert b["n_iter"] == 1
    np.testing.assert_array_equal(a["order"], b["order"])
    np.testing.assert_allclose(a["phi"], b["phi"], rtol=1e-14)


def test_permutation_invariance():
    pop = synth.single_halo()
    p = O.Params()
    a = O.unbind_population(pop, p)[0]
    rng = np.random.default_rng(0)
    perm = rng.permutation(pop.n_particles)
    q = copy.copy(pop)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        setattr(q, k, getattr(pop, k)[perm])
    b = O.unbind_population(q, p)[0]
    np.testing.assert_array_equal(perm[b["bound_idx"]], a["bound_idx"])
    np.testing.assert_allclose(b["phi"], a["phi"], rtol=1e-12)
    assert b["r_vir"] == pytest.approx(a["r_vir"], rel=1e-14)


def test_galilean_invariance():
    pop = synth.single_halo()
    p = O.Params()
    a = O.unbind_population(pop, p)[0]
    q = copy.copy(pop)
    q.vx, q.vy, q.vz = pop.vx + 250.0, pop.vy - 400.0, pop.vz + 1000.0
    b = O.unbind_population(q, p)[0]
    np.testing.assert_array_equal(a["bound_idx"], b["bound_idx"])
    np.testing.assert_allclose(b["vbulk"] - a["vbulk"], [250.0, -400.0, 1000.0], rtol=1e-10)


def test_periodic_translation_invariance():
    # Sect. 3.2: shifting all particles (with periodic wrap) leaves the
    # result unchanged.
    small = synth.halo_batch(seed=99, n_halos=1, n_lo=3000, n_hi=3000, coord_type=synth.COORD_F64)
    box = 1000.0
    base = copy.copy(small)
    base.box = box
    base.centre = np.array([[995.0, 3.0, 500.0]])
    rel = [small.x - small.centre[0, 0], small.y - small.centre[0, 1], small.z - small.centre[0, 2]]
    base.x, base.y, base.z = [np.mod(rel[i] + base.centre[0, i], box) for i in range(3)]
    p = O.Params()
    a = O.unbind_population(base, p)[0]
    shift = np.array([17.25, -600.5, 333.0])
    q = copy.copy(base)
    q.x, q.y, q.z = [np.mod(getattr(base, k) + shift[i], box) for i, k in enumerate("xyz")]
    q.centre = np.mod(base.centre + shift, box)
    b = O.unbind_population(q, p)[0]
    np.testing.assert_array_equal(a["bound_idx"], b["bound_idx"])
    np.testing.assert_allclose(a["phi"], b["phi"], rtol=1e-9)
    # and identical to the non-periodic, unwrapped halo
    c = O.unbind_population(small, p)[0]
    np.testing.assert_array_equal(a["bound_idx"], c["bound_idx"])


def _halo_arrays(r, v, m):
    n = r.shape[0]
    d = np.zeros((n, 3))
    d[:, 0] = r
    return d, v, m, np.ones(n, bool)


def test_single_particle():
    p = O.Params(H=0.0)
    d, v, m, ins = _halo_arrays(np.array([3.0]), np.array([[10.0, 0, 0]]), np.array([1e10]))
    o = O.unbind_halo(d, v, m, ins, p)       # u = v - v_bulk = 0: bound
    assert o["order"].tolist() == [0] and o["n_iter"] == 1
    assert o["phi"][0] == pytest.approx(-G * 1e10 / 3.0, rel=1e-15)
    p = O.Params(H=0.1)
    o = O.unbind_halo(d, v, m * 1e-6, ins, p)  # Hubble flow 0.3 km/s beats v_esc ~ 0.17
    assert o["status"] & O.EMPTY and o["order"].shape[0] == 0


def test_cold_uniform_sphere_all_bound():
    rng = np.random.default_rng(2)
    n = 5000
    pos, _ = synth.sample_uniform_sphere(rng, n, 50.0, 0.0)
    v = np.tile([[120.0, -30.0, 5.0]], (n, 1))     # all move with the bulk
    o = O.unbind_halo(pos, v, np.full(n, 1e8), np.ones(n, bool), O.Params(H=0.0))
    assert o["n_iter"] == 1 and o["order"].shape[0] == n


def test_all_unbound_gives_empty():
    rng = np.random.default_rng(4)
    n = 1000
    pos, _ = synth.sample_uniform_sphere(rng, n, 50.0, 0.0)
    m = np.full(n, 1e8)
    r = np.sqrt((pos ** 2).sum(1))
    o = np.lexsort((np.arange(n), r))
    phi = np.empty(n)
    phi[o] = O.potential_bruteforce(r[o], m[o], G)
    dirs = rng.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    v = dirs * (10.0 * np.sqrt(2.0 * np.abs(phi)))[:, None]   # |v_bulk| << 9 v_esc
    res = O.unbind_halo(pos, v, m, np.ones(n, bool), O.Params(H=0.0))
    assert res["status"] & O.EMPTY
    assert res["n_iter"] >= 1 and res["order"].shape[0] == 0


def test_hubble_term_cuts_cold_sphere_at_analytic_radius():
    # Cold uniform sphere (v = 0) with a Hubble flow: u = H r, and
    # 2|phi(r)| = G M (3 R^2 - r^2) / R^3.  Particles beyond
    # r* = R sqrt(3 G M / (H^2 R^3 + G M)) are unbound in the first iteration.
    rng = np.random.default_rng(8)
    n, R, mp = 200_000, 100.0, 1e6
    pos, _ = synth.sample_uniform_sphere(rng, n, R, 0.0)
    M = n * mp
    H = 2.0 * math.sqrt(G * M / R ** 3)          # r* = R sqrt(3/5)
    res = O.unbind_halo(pos, np.zeros((n, 3)), np.full(n, mp), np.ones(n, bool), O.Params(H=H))
    r = np.sqrt((pos ** 2).sum(1))
    first = res["removed_iter"] == 1
    r_star = R * math.sqrt(3 * G * M / (H * H * R ** 3 + G * M))
    # the first-iteration cut sits at the analytic radius within sampling noise
    assert abs(r[first].min() / r_star - 1) < 5e-3
    assert abs(r[~first].max() / r_star - 1) < 5e-3


def test_strict_inequality_keeps_marginal_particle():
    # Two unit-mass particles, G = 1, H = 0, at r = 1 and r = 2:
    # phi_1 = -(1 + 1/2) = -1.5, phi_2 = -(1/2 + 1/2) = -1.
    # Velocities -(1,1,0) and +(1,1,0) keep v_bulk = 0 and give |u|^2 = 2
    # exactly: particle 2 sits on the escape speed and stays (strict >).
    d = np.array([[1.0, 0, 0], [2.0, 0, 0]])
    v = np.array([[-1.0, -1.0, 0], [1.0, 1.0, 0]])
    p = O.Params(G=1.0, H=0.0)
    o = O.unbind_halo(d, v, np.ones(2), np.ones(2, bool), p)
    assert o["order"].tolist() == [0, 1] and o["n_iter"] == 1
    np.testing.assert_allclose(o["phi"], [-1.5, -1.0], rtol=1e-15)
    # a hair faster and it leaves in the first iteration
    v2 = v * (1.0 + 1e-12)
    o = O.unbind_halo(d, v2, np.ones(2), np.ones(2, bool), p)
    assert o["removed_iter"].tolist() == [0, 1]


def test_vbulk_is_mass_weighted():
    d = np.array([[1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0]])
    v = np.array([[0.0, 0, 0], [3.0, 0, 0], [0.0, 6.0, 0]])
    m = np.array([1.0, 2.0, 3.0]) * 1e15
    o = O.unbind_halo(d, v, m, np.ones(3, bool), O.Params(H=0.0))
    np.testing.assert_allclose(o["vbulk"], [1.0, 3.0, 0.0], rtol=1e-15)
    # The loop's bulk velocity is mass weighted too.  G = 1, H = 0: a heavy
    # particle (m = 100, r = 1, at rest) and two light ones (m = 1, r = 2, 3)
    # moving at w = 11 along x.  v_bulk = 22/102, so u = 11 (1 - 2/102) = 10.78
    # and u^2 = 116.3 exceeds 2|phi| = 2 (50 + 1/2 + 1/3) = 101.7 and
    # 2 (101/3 + 1/3) = 68: both light particles leave in iteration 1.
    # (An unweighted mean, 22/3, would keep them: u^2 = 13.4.)
    d = np.array([[1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0]])
    v = np.array([[0.0, 0, 0], [11.0, 0, 0], [11.0, 0, 0]])
    o = O.unbind_halo(d, v, np.array([100.0, 1.0, 1.0]), np.ones(3, bool), O.Params(G=1.0, H=0.0))
    assert o["removed_iter"].tolist() == [0, 1, 1]


def test_gather_sphere_and_minimum_image():
    pop = synth.single_halo()
    q = copy.copy(pop)
    q.radius = np.array([50.0])
    pidx, d, v, m, inside = O.gather_sphere(q, 0)
    r = np.sqrt((d ** 2).sum(1))
    assert np.all(r[inside] <= 50.0) and np.all(r[~inside] > 50.0)
    d2 = O.recentre(np.array([999.0, 1.0]), np.array([0.0, 0.0]), np.array([0.0, 0.0]),
                    np.array([1.0, 0.0, 0.0]), 1000.0)
    np.testing.assert_allclose(d2[:, 0], [-2.0, 0.0])


def test_profile_counts_and_mass():
    pop = synth.single_halo()
    res = O.unbind_population(pop, O.Params(), n_bins=20, r_min_frac=0.01)[0]
    prof = res["profile"]
    r = res["r"]
    edges = res["r_vir"] * 0.01 ** (1 - np.arange(21) / 20)
    for b in range(20):
        n_b = int(np.sum((r > edges[b]) & (r <= edges[b + 1])))
        assert prof[b, 0] == n_b
    assert prof[-1, 1] == pytest.approx(res["m_vir"], rel=1e-12)
    assert prof[-1, 3] == pytest.approx(math.sqrt(G * res["m_vir"] / res["r_vir"]), rel=1e-12)
    shell = prof[:, 0] * pop.m0 / (4 * math.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3))
    np.testing.assert_allclose(prof[:, 2], shell, rtol=1e-12)


def test_infall_cancelling_hubble_flow_stays_bound():
    # A cold sphere whose particles fall in at exactly the Hubble rate,
    # v = -H d, has u = v - v_bulk + H d = 0: nothing is removed even with a
    # Hubble constant that would unbind the static sphere.
    rng = np.random.default_rng(12)
    n, R, mp = 4000, 100.0, 1e6
    pos, _ = synth.sample_uniform_sphere(rng, n, R, 0.0)
    pos -= pos.mean(0)
    H = 3.0 * math.sqrt(G * n * mp / R ** 3)
    o = O.unbind_halo(pos, -H * pos, np.full(n, mp), np.ones(n, bool), O.Params(H=H))
    assert o["n_iter"] == 1 and o["order"].shape[0] == n
    o = O.unbind_halo(pos, np.zeros((n, 3)), np.full(n, mp), np.ones(n, bool), O.Params(H=H))
    assert o["order"].shape[0] < n


def test_radius_order_matters():
    # Two haloes with identical radii multiset but different mass order must
    # give phi from the radially sorted list (Appendix A): heavy particle
    # inside vs outside changes phi of the other particle.
    r = np.array([1.0, 2.0])
    a = O.potential_sorted(r, np.array([10.0, 1.0]), 1.0)
    b = O.potential_sorted(r, np.array([1.0, 10.0]), 1.0)
    np.testing.assert_allclose(a, [-(10.0 + 0.5), -(10.0 / 2 + 0.5)])
    np.testing.assert_allclose(b, [-(1.0 + 5.0), -(1.0 / 2 + 5.0)])


def test_profile_two_bins_hand_worked():
    # Six particles at r = 1, 2, 3, 4, 5, 8 with masses 1..6, G = 1,
    # r_out = 8, two bins from f = 1/4: edges e_0 = 8 (1/4)^1 = 2,
    # e_1 = 8 (1/4)^(1/2) = 4, e_2 = 8.  Bin 0 = (2, 4] holds r = 3, 4
    # (r = 2 sits on e_0 and stays out): count 2, shell mass 3 + 4 = 7,
    # M(<= 4) = 1 + 2 + 3 + 4 = 10, density 7 / (4 pi / 3 (4^3 - 2^3))
    # = 21 / (224 pi), v_c = sqrt(10 / 4).  Bin 1 = (4, 8] holds r = 5, 8:
    # count 2, shell mass 11, M(<= 8) = 21, density 11 / (4 pi / 3 (8^3 - 4^3))
    # = 33 / (1792 pi), v_c = sqrt(21 / 8).
    r = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 8.0])
    m = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    want = np.array([[2.0, 10.0, 0.029841551829730376, 1.5811388300841898],
                     [2.0, 21.0, 0.005861733395125609, 1.620185174601965]])
    np.testing.assert_allclose(O.profile(r, m, 8.0, 2, 0.25, 1.0), want, rtol=1e-14)
    # r_vir = 0: the outermost particle (8) is r_out, the same rows
    np.testing.assert_allclose(O.profile(r, m, 0.0, 2, 0.25, 1.0), want, rtol=1e-14)
    # r_vir = 4: edges 1, 2, 4; bin 0 = (1, 2] holds r = 2 (mass 2), M(<= 2) = 3,
    # density 2 / (4 pi / 3 (2^3 - 1)) = 3 / (14 pi), v_c = sqrt(3 / 2);
    # bin 1 = (2, 4] as above with G M / r = 10 / 4
    want4 = np.array([[1.0, 3.0, 0.06820926132509800, 1.2247448713915890],
                      [2.0, 10.0, 0.029841551829730376, 1.5811388300841898]])
    np.testing.assert_allclose(O.profile(r, m, 4.0, 2, 0.25, 1.0), want4, rtol=1e-14)

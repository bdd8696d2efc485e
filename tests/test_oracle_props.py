"""Pins of the oracle's integral properties (spin parameter, energies,
rotation-curve peak; Sect. 3.1) and of its catalogue cross-identification
(xi = N_shared^2 / (N_1 N_2), Sect. 3.2): a hand-worked two-particle case,
closed forms, exact identities, invariances and special cases."""
import math

import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import synth


def _props(d, v, m, H=0.0, k_vir=-1):
    prm = O.Params(H=H)
    r = np.sqrt((d * d).sum(axis=1))
    order = np.lexsort((np.arange(len(r)), r))
    phi = O.potential_sorted(r[order], m[order], prm.G)
    return O.halo_properties(d[order], v[order], m[order], phi, k_vir, prm), prm


def test_two_particle_worked_example():
    # two masses m at (+-a, 0, 0) moving (0, +-w, 0), H = 0.  By hand:
    #   phi = -G (m/a + m/a) for both (equal radii), U = (1/2) 2 m phi = -2 G m^2 / a
    #   J = 2 m a w along z, K = m w^2, E = K + U, M = 2 m
    #   lambda = J sqrt|E| / (G M^2.5)
    #   v_c: the outer of the tied pair encloses 2 m: v_max = sqrt(2 G m / a) at a
    m, a, w, G = 1e10, 100.0, 50.0, 4.3009e-6
    d = np.array([[a, 0.0, 0.0], [-a, 0.0, 0.0]])
    v = np.array([[0.0, w, 0.0], [0.0, -w, 0.0]])
    p, _ = _props(d, v, np.array([m, m]))
    K, U, Jz = 2.5e13, -8.6018e12, 1e14
    E = K + U                                         # 1.63982e13
    lam = Jz * math.sqrt(E) / (G * (2e10) ** 2.5)     # 1.66443...
    assert p["n"] == 2 and p["M"] == 2e10
    np.testing.assert_allclose(p["J"], [0.0, 0.0, Jz], rtol=1e-14, atol=1e-3)
    assert p["K"] == pytest.approx(K, rel=1e-14)
    assert p["U"] == pytest.approx(U, rel=1e-14)
    assert p["E"] == pytest.approx(E, rel=1e-13)
    assert p["lam"] == pytest.approx(1.66443, rel=1e-5) and p["lam"] == pytest.approx(lam, rel=1e-13)
    assert p["v_max"] == pytest.approx(math.sqrt(2 * G * m / a), rel=1e-14) and p["r_max"] == a


def _mirrored_sphere(n, R, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d *= (R * rng.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    return np.concatenate([d, -d])


def test_solid_body_rotation():
    # v = omega x d on a sphere mirrored through the centre (sum m d = 0,
    # v_bar = 0 exactly): J = sum m (|d|^2 omega - (d . omega) d) (the triple
    # product expanded), K = omega J_z / 2 identically, J_z -> 2/5 M R^2 omega
    R, om, n = 100.0, 0.5, 20000
    d = _mirrored_sphere(n, R, 3)
    v = np.cross(np.array([0.0, 0.0, om]), d)
    m = np.full(d.shape[0], 1e8)
    p, _ = _props(d, v, m)
    M = m.sum()
    assert p["K"] == pytest.approx(0.5 * om * p["J"][2], rel=1e-12)
    assert p["J"][2] == pytest.approx(0.4 * M * R * R * om, rel=0.02)
    J_inertia = om * np.array([-(m * d[:, 0] * d[:, 2]).sum(), -(m * d[:, 1] * d[:, 2]).sum(),
                               (m * (d[:, 0] ** 2 + d[:, 1] ** 2)).sum()])
    np.testing.assert_allclose(p["J"], J_inertia, rtol=1e-10, atol=1e-10 * abs(J_inertia[2]))


def test_uniform_sphere_energy_and_rotation_curve():
    # U -> -3/5 G M^2 / R; v_c rises to the edge: v_max = sqrt(G M / r_N) at r_N
    R, n = 100.0, 50000
    d = _mirrored_sphere(n // 2, R, 4)
    m = np.full(d.shape[0], 1e7)
    p, prm = _props(d, np.zeros_like(d), m)
    M = m.sum()
    assert p["U"] == pytest.approx(-0.6 * prm.G * M * M / R, rel=0.02)
    r_last = np.sqrt((d * d).sum(axis=1)).max()
    assert p["r_max"] == r_last and p["v_max"] == pytest.approx(math.sqrt(prm.G * M / r_last), rel=1e-14)
    assert p["K"] == 0.0 and p["lam"] == 0.0


def test_nfw_rotation_curve_peak():
    # untruncated NFW: v_c peaks at x = 2.163 r_s, v_max^2 = G M(<r_max) / r_max
    c, r200, n = 8.0, 200.0, 200000
    rng = np.random.default_rng(5)
    d, _ = synth.sample_nfw(rng, n, c, r200)
    m = np.full(n, 1e7)
    p, prm = _props(d, np.zeros_like(d), m)
    rs = r200 / c
    x_t = 2.0 * c
    mfun = lambda x: math.log(1 + x) - x / (1 + x)
    x_pk = 2.16258
    assert p["r_max"] / rs == pytest.approx(x_pk, rel=0.15)
    v_pk = math.sqrt(prm.G * m.sum() * mfun(x_pk) / mfun(x_t) / (x_pk * rs))
    assert p["v_max"] == pytest.approx(v_pk, rel=0.01)


def test_invariances_and_virial_selection():
    rng = np.random.default_rng(6)
    d = rng.normal(0, 50, (3000, 3))
    v = rng.normal(0, 80, (3000, 3)) + np.cross([0.0, 0.0, 0.3], d)
    m = rng.uniform(1e8, 3e8, 3000)
    p, _ = _props(d, v, m, H=0.1)
    # Galilean boost: nothing changes (v_bar absorbs it)
    q, _ = _props(d, v + np.array([300.0, -200.0, 50.0]), m, H=0.1)
    for k in ("K", "U", "lam", "v_max"):
        assert q[k] == pytest.approx(p[k], rel=1e-10)
    np.testing.assert_allclose(q["J"], p["J"], rtol=1e-9, atol=1e-6 * np.abs(p["J"]).max())
    # rotation: |J|, K, U, lambda unchanged, J rotated
    a = 0.7
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])
    Rx = np.array([[1.0, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    Q = Rx @ Rz
    q, _ = _props(d @ Q.T, v @ Q.T, m, H=0.1)
    for k in ("K", "U", "lam", "v_max", "r_max"):
        assert q[k] == pytest.approx(p[k], rel=1e-10)
    np.testing.assert_allclose(q["J"], Q @ p["J"], rtol=1e-9, atol=1e-9 * np.abs(p["J"]).max())
    # the virial selection uses the first k_vir + 1 particles only
    r = np.sqrt((d * d).sum(axis=1))
    order = np.lexsort((np.arange(3000), r))
    prm = O.Params(H=0.1)
    phi = O.potential_sorted(r[order], m[order], prm.G)
    s = O.halo_properties(d[order], v[order], m[order], phi, 999, prm)
    t = O.halo_properties(d[order][:1000], v[order][:1000], m[order][:1000], phi[:1000], -1, prm)
    assert s["n"] == 1000 and s["M"] == t["M"] and s["lam"] == t["lam"]


def test_match_catalogs_cases():
    A = [np.arange(0, 100), np.arange(100, 150), np.arange(150, 160)]
    # identical catalogues: every halo matches itself with xi = 1
    best, shared, xi = O.match_catalogs(A, A)
    assert best.tolist() == [0, 1, 2] and shared.tolist() == [100, 50, 10] and np.all(xi == 1.0)
    # the first halo split in two halves: xi = (N/2)^2 / (N N/2) = 1/2 each; ties
    # go to the lower index
    B = [np.arange(0, 50), np.arange(50, 100), np.arange(100, 150)]
    best, shared, xi = O.match_catalogs(A, B)
    assert best.tolist() == [0, 2, -1] and shared.tolist() == [50, 50, 0]
    assert xi.tolist() == [0.5, 1.0, 0.0]
    # a permuted second catalogue permutes the answers
    perm = [2, 0, 1]
    Bp = [B[k] for k in perm]
    best_p, _, xi_p = O.match_catalogs(A, Bp)
    inv = {old: new for new, old in enumerate(perm)}
    assert best_p.tolist() == [inv[0], inv[2], -1] and xi_p.tolist() == xi.tolist()
    # 30 of 40 shared with a 60-particle halo, 10 with a 10-particle one:
    # xi = 900 / 2400 = 0.375 against 100 / 400 = 0.25
    A2 = [np.arange(0, 40)]
    B2 = [np.arange(-30, 30), np.arange(30, 40)]
    best, shared, xi = O.match_catalogs(A2, B2)
    assert best.tolist() == [0] and shared.tolist() == [30] and xi[0] == pytest.approx(0.375)

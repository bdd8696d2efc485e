"""CPU: the synthetic inputs follow the stated recipes of the workloads.

The generator stands in for the paper's N-body snapshots, so its
distributions are checked here against independently computed references:
the truncated NFW radial distribution by quadrature of the density (not the
closed-form enclosed mass the generator uses), the particle-count law by
quadrature of N_p^-1.9, the printed value of the critical density, and
Kolmogorov-Smirnov statistics at a fixed seed.
"""
import math

import numpy as np
import pytest

from paper_0904_3662_gb300 import synth

integrate = pytest.importorskip("scipy.integrate")
stats = pytest.importorskip("scipy.stats")


def _ks(sample, cdf):
    """Kolmogorov-Smirnov distance of a sample from a CDF given on the sample."""
    x = np.sort(np.asarray(sample, dtype=np.float64))
    f = np.array([cdf(v) for v in x])
    n = x.shape[0]
    i = np.arange(1, n + 1)
    return max(np.max(i / n - f), np.max(f - (i - 1) / n))


def _nfw_cdf(c, x_t):
    """Enclosed-mass fraction of an NFW sphere truncated at x_t = r_t / r_s,
    by quadrature of rho(x) x^2 ~ x / (1 + x)^2."""
    norm = integrate.quad(lambda x: x / (1.0 + x) ** 2, 0.0, x_t)[0]
    return lambda x: integrate.quad(lambda t: t / (1.0 + t) ** 2, 0.0, min(x, x_t))[0] / norm


def test_critical_density_and_r200_of_the_stated_units():
    # rho_crit = 3 H^2 / (8 pi G) = 277.54 (Msun/h)/(kpc/h)^3, 200 rho_crit = 55,508
    assert abs(synth.RHO_CRIT - 277.54) < 0.01
    assert abs(synth.DELTA_RHO_200C - 55508.0) < 1.0
    # M(<R_200) = 200 rho_crit 4 pi R_200^3 / 3 for the 1e12 Msun/h halo
    r = synth.r200_of_mass(1e12)
    assert abs(200.0 * 277.54 * 4.0 * math.pi * r ** 3 / 3.0 / 1e12 - 1.0) < 1e-4


def test_single_halo_recipe():
    pop = synth.single_halo()
    assert pop.n_particles == 11_000 and pop.n_halos == 1
    assert pop.coord_type == synth.COORD_F64 and pop.x.dtype == np.float64
    r200 = synth.r200_of_mass(1e12)
    assert abs(pop.radius[0] - 2.0 * r200) < 1e-9 and abs(pop.r200[0] - r200) < 1e-9
    d = np.stack([pop.x, pop.y, pop.z], 1) - pop.centre[0][None, :]
    r = np.sqrt((d * d).sum(1))
    assert r.max() <= pop.radius[0] * (1.0 + 1e-12)
    # 10,000 particles of the c = 10 profile truncated at 2 R_200 (x_t = 20;
    # M_200 and c fix r_s = R_200 / c = 16.3 kpc/h) and 1,000 uniform in the
    # same sphere; the KS distance of all 11,000 radii at the 0.1 % level
    rs = r200 / 10.0
    f_nfw = _nfw_cdf(10.0, 20.0)
    cdf = lambda v: (10_000 * f_nfw(v / rs) + 1_000 * min(v / (2.0 * r200), 1.0) ** 3) / 11_000
    assert _ks(r, cdf) < 1.95 / math.sqrt(r.shape[0])
    # the uniform background carries N(0, 600 km/s) components: the 500
    # fastest particles are almost all of it
    v = np.sqrt(pop.vx ** 2 + pop.vy ** 2 + pop.vz ** 2)
    fast = np.sort(v)[-500:]
    assert np.median(fast) > 900.0
    # total mass of the NFW component within R_200 is 1e12 Msun/h
    n_in = 10_000 * f_nfw(10.0)
    assert abs(n_in * pop.m0 / 1e12 - 1.0) < 1e-3


def _member_counts(count, frac=0.15):
    """N_p of each halo from its candidate count N_p + rint(frac N_p)."""
    n = np.rint(count / (1.0 + frac)).astype(np.int64)
    for k in range(n.shape[0]):
        for dn in (0, -1, 1, -2, 2):
            if n[k] + dn + int(np.rint(frac * (n[k] + dn))) == count[k]:
                n[k] += dn
                break
        else:
            raise AssertionError(f"count {count[k]} is not N + rint({frac} N)")
    return n


def test_batch_counts_follow_the_power_law_and_contaminant_fraction():
    pop = synth.halo_batch(n_halos=2000)
    assert pop.n_halos == 2000 and pop.coord_type == synth.COORD_F32_REL
    n_p = _member_counts(pop.count)
    assert n_p.min() >= 100 and n_p.max() <= 100_000
    lo, hi = 100.0, 100_000.0
    norm = integrate.quad(lambda t: t ** -1.9, lo, hi)[0]
    # CDF by quadrature; integer rounding moves a draw by < 0.5 (tiny against 1/N)
    cdf = lambda v: integrate.quad(lambda t: t ** -1.9, lo, min(max(v, lo), hi))[0] / norm
    assert _ks(n_p, cdf) < 1.95 / math.sqrt(2000)        # KS at the 0.1 % level
    assert np.all(pop.count == n_p + np.rint(0.15 * n_p).astype(np.int64))
    assert 1_700_000 < pop.n_particles < 1_900_000


def test_batch_concentrations_are_lognormal():
    pop = synth.halo_batch(n_halos=2000)
    lc = np.log(pop.conc)
    assert abs(lc.mean() - math.log(10.0)) < 3.0 * 0.25 / math.sqrt(2000)
    assert abs(lc.std() - 0.25) < 0.02
    assert stats.kstest((lc - math.log(10.0)) / 0.25, "norm").pvalue > 0.01


def test_batch_positions_are_float32_relative_and_inside_the_sphere():
    pop = synth.halo_batch(seed=synth.SEED_BASE + 61, n_halos=50, n_lo=100, n_hi=3000)
    assert pop.x.dtype == np.float32 and np.all(pop.centre == 0.0)
    for h in range(pop.n_halos):
        s = slice(int(pop.offset[h]), int(pop.offset[h] + pop.count[h]))
        r = np.sqrt(pop.x[s].astype(np.float64) ** 2 + pop.y[s] ** 2.0 + pop.z[s] ** 2.0)
        assert r.max() <= pop.radius[h] * (1.0 + 1e-6)
        # the sphere is 2 R_200 of the halo's own NFW mass N_p m_p m(c) / m(2c)
        n_p = _member_counts(pop.count[h:h + 1])[0]
        c = pop.conc[h]
        f = _nfw_cdf(c, 2.0 * c)
        m200 = n_p * synth.PARTICLE_MASS * f(c)
        assert abs(synth.r200_of_mass(m200) / pop.r200[h] - 1.0) < 1e-6


def test_generators_are_seeded():
    a = synth.halo_batch(seed=5, n_halos=20, n_lo=100, n_hi=2000)
    b = synth.halo_batch(seed=5, n_halos=20, n_lo=100, n_hi=2000)
    c = synth.halo_batch(seed=6, n_halos=20, n_lo=100, n_hi=2000)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.vz, b.vz) and np.array_equal(a.count, b.count)
    assert not np.array_equal(a.count, c.count)


def test_nfw_velocities_follow_the_jeans_dispersion():
    # isotropic Jeans equation of the truncated profile with rho sigma^2 = 0
    # at the truncation radius, by quadrature: rho(r) sigma^2(r) =
    # int_r^{r_t} rho(r') G M(r') / r'^2 dr', M from the density by quadrature
    rng = np.random.default_rng(synth.SEED_BASE + 62)
    c, r200 = 10.0, synth.r200_of_mass(1e12)
    rs, x_t = r200 / c, 2.0 * c
    pos, vel = synth.sample_nfw(rng, 200_000, c, r200)
    shape = lambda x: 1.0 / (x * (1.0 + x) ** 2)
    i_c = integrate.quad(lambda t: t / (1.0 + t) ** 2, 0.0, c)[0]
    rho_s = 1e12 / (4.0 * math.pi * rs ** 3 * i_c)              # M(<R_200) = 1e12
    mass = lambda x: 4.0 * math.pi * rho_s * rs ** 3 * integrate.quad(lambda t: t / (1.0 + t) ** 2, 0.0, x)[0]
    g = synth.G_GRAV
    x = np.sqrt((pos * pos).sum(1)) / rs
    for xc in (0.3, 1.0, 3.0, 8.0):
        sel = np.abs(np.log(x / xc)) < 0.05
        sig2 = integrate.quad(lambda t: shape(t) * g * mass(t) / (t * rs) ** 2 * rs, xc, x_t, limit=200)[0] / shape(xc)
        got = float((vel[sel] ** 2).sum(1).mean() / 3.0)
        n = int(sel.sum())
        # sampling error of a variance from 3n Gaussian components, plus the
        # variation of sigma^2 across the +-5 % shell
        assert abs(got / sig2 - 1.0) < 4.0 * math.sqrt(2.0 / (3 * n)) + 0.01, (xc, got, sig2, n)

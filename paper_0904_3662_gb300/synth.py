"""Seeded synthetic halo populations (input generation only).

Nothing in this module performs any step of the unbinding method: it draws
particles.  It is the one module that both the CUDA path (tests, bench) and
the CPU oracle consume, so it deliberately holds no potential, escape-velocity
or virial-radius arithmetic.

Physical model of the inputs (a stand-in for the paper's N-body snapshots,
which are not available):

* Haloes are truncated NFW spheres.  Radii follow the enclosed-mass CDF
  m(x)/m(x_t), m(x) = ln(1+x) - x/(1+x), x = r/r_s, truncated at x_t = 2c
  (twice R_200).  Directions are isotropic.
* Velocities are isotropic Gaussians whose dispersion solves the spherical
  Jeans equation of the truncated profile with rho*sigma^2 = 0 at the
  truncation radius (evaluated by quadrature on a log grid).
* Contaminants are uniform in the gather sphere with N(0, 600 km/s) velocity
  components: mostly unbound particles.
* Units: kpc/h, km/s, Msun/h; G = 4.3009e-6 kpc (km/s)^2 / Msun,
  H0 = 0.1 h km/s per kpc/h, so rho_crit = 3 H0^2 / (8 pi G).

The five workloads are the single halo, the 2,000-halo batch, the
large-halo tail in a periodic box, the 1e5-halo precision sweep and the
serving stream; the small variants keep the same structure at sizes a CPU
oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G_GRAV = 4.3009e-6          # kpc (km/s)^2 / Msun
H0 = 0.1                    # h km/s per kpc/h  (100 km/s/Mpc)
RHO_CRIT = 3.0 * H0 * H0 / (8.0 * math.pi * G_GRAV)   # (Msun/h) / (kpc/h)^3
DELTA_RHO_200C = 200.0 * RHO_CRIT

COORD_F64 = 0
COORD_F32_REL = 1
COORD_F32_BOX = 2

SEED_BASE = 20090400


def m_nfw(x):
    """Dimensionless NFW enclosed mass m(x) = ln(1+x) - x/(1+x)."""
    x = np.asarray(x, dtype=np.float64)
    return np.log1p(x) - x / (1.0 + x)


def r200_of_mass(m200):
    """R_200c of a halo of mass M_200c."""
    return (3.0 * m200 / (4.0 * math.pi * DELTA_RHO_200C)) ** (1.0 / 3.0)


# Particle mass shared by all workloads: a c = 10, 1e12 Msun/h halo sampled
# with 1e4 particles out to 2 R_200.
PARTICLE_MASS = 1e12 * float(m_nfw(20.0)) / float(m_nfw(10.0)) / 1e4


class _NFWTables:
    """Inverse-CDF and Jeans-dispersion tables of a truncated NFW profile."""

    def __init__(self, c: float, x_t: float, n: int = 2048):
        xg = np.geomspace(1e-7 * x_t, x_t, n)
        self.x = xg
        self.cdf = m_nfw(xg) / m_nfw(x_t)
        # Jeans: sigma^2(x) = x (1+x)^2 * int_x^{x_t} m(x') / (x'^3 (1+x')^2) dx'
        # in units of G M_s / r_s.  Trapezoid in ln x from the outer edge in.
        f = m_nfw(xg) / (xg ** 3 * (1.0 + xg) ** 2) * xg   # integrand * x (d ln x)
        lnx = np.log(xg)
        seg = 0.5 * (f[1:] + f[:-1]) * np.diff(lnx)
        tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
        self.sig2 = xg * (1.0 + xg) ** 2 * tail

    def radii(self, u):
        return np.interp(u, self.cdf, self.x)

    def sigma2(self, x):
        return np.interp(x, self.x, self.sig2)


def _iso_dirs(rng, n):
    cth = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(ph), sth * np.sin(ph), cth], axis=1)


def sample_nfw(rng, n, c, r200, trunc=2.0):
    """n particles of a c-concentration NFW halo truncated at trunc*R_200.

    Returns (pos, vel) as float64 arrays of shape (n, 3), relative to the
    halo centre and at rest in its frame."""
    rs = r200 / c
    x_t = trunc * c
    tab = _NFWTables(c, x_t)
    x = tab.radii(rng.uniform(0.0, 1.0, n))
    pos = _iso_dirs(rng, n) * (x * rs)[:, None]
    m200 = 4.0 * math.pi * DELTA_RHO_200C * r200 ** 3 / 3.0
    ms = m200 / float(m_nfw(c))
    sig = np.sqrt(np.maximum(tab.sigma2(x), 0.0) * G_GRAV * ms / rs)
    vel = rng.standard_normal((n, 3)) * sig[:, None]
    return pos, vel


def sample_uniform_sphere(rng, n, radius, sigma_v):
    """n particles uniform in a sphere with N(0, sigma_v) velocity components."""
    rr = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = _iso_dirs(rng, n) * rr[:, None]
    vel = rng.standard_normal((n, 3)) * sigma_v
    return pos, vel


def powerlaw_counts(rng, n, lo, hi, slope=-1.9):
    """Integer counts drawn from dN/dN_p ~ N_p^slope on [lo, hi]."""
    a = slope + 1.0
    u = rng.uniform(0.0, 1.0, n)
    v = (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


@dataclasses.dataclass
class Population:
    """A batch of haloes in one SoA particle store.

    Particle arrays hold all haloes back to back; halo h owns the candidate
    slice [offset[h], offset[h] + count[h]).  Coordinates are stored in the
    precision that coord_type names; mass is None when every particle
    carries m0."""
    name: str
    coord_type: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray | None
    m0: float
    box: float
    centre: np.ndarray          # (H, 3) float64
    radius: np.ndarray          # (H,)   float64
    offset: np.ndarray          # (H,)   int64
    count: np.ndarray           # (H,)   int64
    r200: np.ndarray            # (H,)   float64, generator metadata
    conc: np.ndarray            # (H,)   float64, generator metadata
    u_th: np.ndarray | None = None   # specific thermal energy (km/s)^2 of gas particles, 0 elsewhere

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_halos(self) -> int:
        return int(self.offset.shape[0])


def _alloc(n, dtype):
    return [np.empty(n, dtype=dtype) for _ in range(6)]


def _halo_block(rng, n_nfw, n_cont, c, m_p, cont_sigma=600.0):
    """One NFW halo plus uniform contaminants in its 2 R_200 sphere, shuffled."""
    m200 = n_nfw * m_p * float(m_nfw(c)) / float(m_nfw(2.0 * c))
    r200 = r200_of_mass(m200)
    p1, v1 = sample_nfw(rng, n_nfw, c, r200)
    if n_cont > 0:
        p2, v2 = sample_uniform_sphere(rng, n_cont, 2.0 * r200, cont_sigma)
        p1 = np.concatenate([p1, p2])
        v1 = np.concatenate([v1, v2])
    perm = rng.permutation(p1.shape[0])
    return p1[perm], v1[perm], r200


def single_halo(seed=SEED_BASE + 1, n_nfw=10_000, n_cont=1_000, c=10.0,
                m200=1e12, centre=(31250.125, 47811.5, 12007.75)):
    """One truncated NFW halo (M_200c and c primary, r_s = R_200/c) plus a
    uniform, mostly unbound background; float64 positions in kpc/h."""
    rng = np.random.default_rng(seed)
    m_p = m200 * float(m_nfw(2.0 * c)) / float(m_nfw(c)) / n_nfw
    r200 = r200_of_mass(m200)
    p1, v1 = sample_nfw(rng, n_nfw, c, r200)
    p2, v2 = sample_uniform_sphere(rng, n_cont, 2.0 * r200, 600.0)
    pos = np.concatenate([p1, p2])
    vel = np.concatenate([v1, v2])
    perm = rng.permutation(pos.shape[0])
    pos = pos[perm] + np.asarray(centre)[None, :]
    vel = vel[perm]
    n = pos.shape[0]
    return Population(
        name="single_nfw_10k_bg_1k_f64", coord_type=COORD_F64,
        x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
        vx=vel[:, 0].copy(), vy=vel[:, 1].copy(), vz=vel[:, 2].copy(),
        m=None, m0=m_p, box=0.0,
        centre=np.asarray([centre], dtype=np.float64),
        radius=np.asarray([2.0 * r200]), offset=np.zeros(1, np.int64),
        count=np.asarray([n], np.int64), r200=np.asarray([r200]),
        conc=np.asarray([c]))


def halo_batch(seed=SEED_BASE + 2, n_halos=2000, n_lo=100, n_hi=100_000,
               cont_frac=0.15, coord_type=COORD_F32_REL, name=None,
               with_masses=False, c_sigma=0.25):
    """Haloes with N_p ~ N_p^-1.9 on [n_lo, n_hi], c ~ lognormal(ln 10, c_sigma),
    plus cont_frac contaminants each.  COORD_F32_REL stores float32 positions
    relative to each centre (centre = 0); COORD_F64 stores float64 positions
    around centres spread over a 1e5 kpc/h region."""
    rng = np.random.default_rng(seed)
    counts = powerlaw_counts(rng, n_halos, n_lo, n_hi)
    conc = np.exp(rng.normal(math.log(10.0), c_sigma, n_halos))
    n_cont = np.rint(cont_frac * counts).astype(np.int64)
    tot = counts + n_cont
    offset = np.concatenate([[0], np.cumsum(tot)[:-1]]).astype(np.int64)
    n = int(tot.sum())
    dt = np.float64 if coord_type == COORD_F64 else np.float32
    x, y, z, vx, vy, vz = _alloc(n, dt)
    m = np.empty(n, dtype=dt) if with_masses else None
    centres = np.zeros((n_halos, 3))
    if coord_type == COORD_F64:
        centres = rng.uniform(0.0, 1e5, (n_halos, 3))
    r200 = np.empty(n_halos)
    for h in range(n_halos):
        p, v, r2 = _halo_block(rng, int(counts[h]), int(n_cont[h]), conc[h], PARTICLE_MASS)
        r200[h] = r2
        s = slice(offset[h], offset[h] + tot[h])
        p = p + centres[h][None, :]
        x[s], y[s], z[s] = p[:, 0], p[:, 1], p[:, 2]
        vx[s], vy[s], vz[s] = v[:, 0], v[:, 1], v[:, 2]
        if m is not None:
            # multi-mass: log-uniform masses over a decade around m_p
            m[s] = PARTICLE_MASS * np.exp(rng.uniform(-1.15, 1.15, tot[h]))
    return Population(
        name=name or f"batch_{n_halos}_nfw_{n_lo}-{n_hi}_cont{int(cont_frac*100)}",
        coord_type=coord_type, x=x, y=y, z=z, vx=vx, vy=vy, vz=vz,
        m=m, m0=PARTICLE_MASS, box=0.0, centre=centres,
        radius=2.0 * r200, offset=offset, count=tot.astype(np.int64),
        r200=r200, conc=conc)


def large_tail(seed=SEED_BASE + 3, n_halos=64, n_lo=1_000_000, n_hi=10_000_000,
               n_sub=20, sub_frac=0.005, box=5e5, host_sigma_v=300.0, counts=None):
    """Massive hosts in a periodic box: N_p ~ N_p^-1.9 on [n_lo, n_hi], each with
    n_sub NFW subhaloes of sub_frac of the host's particles placed at radii drawn
    from the host profile inside R_200 with N(0, 300 km/s) bulk offsets.
    Float32 box coordinates (wrapped into [0, box)).  `counts` (one particle
    count per host) replaces the power-law draw when given."""
    rng = np.random.default_rng(seed)
    drawn = powerlaw_counts(rng, n_halos, n_lo, n_hi)
    counts = drawn if counts is None else np.asarray(counts, dtype=np.int64)
    n_halos = int(counts.shape[0])
    conc = np.exp(rng.normal(math.log(10.0), 0.25, n_halos))
    offset = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    n = int(counts.sum())
    x, y, z, vx, vy, vz = _alloc(n, np.float32)
    centres = rng.uniform(0.0, box, (n_halos, 3))
    r200 = np.empty(n_halos)
    for h in range(n_halos):
        n_h = int(counts[h])
        n_sub_p = int(sub_frac * n_h)
        n_host = n_h - n_sub * n_sub_p
        c = conc[h]
        m200 = n_host * PARTICLE_MASS * float(m_nfw(c)) / float(m_nfw(2.0 * c))
        r2 = r200_of_mass(m200)
        r200[h] = r2
        ps, vs = [], []
        p, v = sample_nfw(rng, n_host, c, r2)
        ps.append(p)
        vs.append(v)
        tab = _NFWTables(c, c)
        for _ in range(n_sub):
            xs = tab.radii(rng.uniform(0.0, 1.0))
            where = _iso_dirs(rng, 1)[0] * xs * (r2 / c)
            cs = math.exp(rng.normal(math.log(15.0), 0.25))
            # subhalo truncated at its own R_200: all its particles lie inside
            rs2 = r200_of_mass(n_sub_p * PARTICLE_MASS)
            p, v = sample_nfw(rng, n_sub_p, cs, rs2, trunc=1.0)
            ps.append(p + where[None, :])
            vs.append(v + rng.normal(0.0, 300.0, 3)[None, :])
        p = np.concatenate(ps)
        v = np.concatenate(vs)
        perm = rng.permutation(p.shape[0])
        p = np.mod(p[perm] + centres[h][None, :], box)
        v = v[perm] + rng.normal(0.0, host_sigma_v, 3)[None, :]
        s = slice(offset[h], offset[h] + n_h)
        x[s], y[s], z[s] = p[:, 0], p[:, 1], p[:, 2]
        vx[s], vy[s], vz[s] = v[:, 0], v[:, 1], v[:, 2]
        # float32 rounding of a coordinate just below the box edge can land on it
        for a in (x, y, z):
            seg = a[s]
            seg[seg >= np.float32(box)] = np.float32(0.0)
    return Population(
        name=f"tail_{n_halos}_hosts_{n_lo:.0e}-{n_hi:.0e}_sub{n_sub}_box{box:.0e}_f32",
        coord_type=COORD_F32_BOX, x=x, y=y, z=z, vx=vx, vy=vy, vz=vz,
        m=None, m0=PARTICLE_MASS, box=box, centre=centres,
        radius=2.0 * r200, offset=offset, count=counts.astype(np.int64),
        r200=r200, conc=conc)


def precision_sweep(seed=SEED_BASE + 4, n_halos=100_000, n_lo=100, n_hi=100_000):
    """The batch population at 1e5 haloes with float64 inputs and the single
    halo's 10 % background fraction."""
    return halo_batch(seed=seed, n_halos=n_halos, n_lo=n_lo, n_hi=n_hi,
                      cont_frac=0.10, coord_type=COORD_F64,
                      name=f"sweep_{n_halos}_nfw_{n_lo}-{n_hi}_cont10_f64")


def shell_profile_batch(seed=SEED_BASE + 8, n_shells=(25, 100, 1250), rise=True, sigma_v=1.0, rho_shells=None):
    """Haloes whose density profile is designed shell by shell: 16 shells of
    n particles each (one halo per entry of n_shells), shell densities
    falling by 2 per shell to shell 11 and, with rise=True, growing by 1.5
    per shell beyond it (a subhalo seen against its host's rising
    background); positions uniform in volume within each shell, cold
    velocities, uniform mass.  rho_shells (16 relative densities) replaces
    that design.  The mean density stays far above 200 rho_crit throughout,
    so the virial crossing is never reached inside the set."""
    rng = np.random.default_rng(seed)
    n_h = len(n_shells)
    counts = np.array([16 * n for n in n_shells], dtype=np.int64)
    offset = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    tot = int(counts.sum())
    pos = np.zeros((tot, 3)); vel = np.zeros((tot, 3))
    radius = np.zeros(n_h)
    m0 = PARTICLE_MASS
    for h, n in enumerate(n_shells):
        if rho_shells is not None:
            rho = [1e12 * 0.5 ** 11 * float(x) for x in rho_shells]
        else:
            rho = [1e12 * 0.5 ** s if s <= 11 else 1e12 * 0.5 ** 11 * (1.5 ** (s - 11) if rise else 0.5 ** (s - 11))
                   for s in range(16)]
        r_in = 0.0
        parts = []
        for s in range(16):
            r_out = (r_in ** 3 + 3.0 * n * m0 / (4.0 * math.pi * rho[s])) ** (1.0 / 3.0)
            rr = (r_in ** 3 + (r_out ** 3 - r_in ** 3) * rng.uniform(0.0, 1.0, n)) ** (1.0 / 3.0)
            parts.append(_iso_dirs(rng, n) * rr[:, None])
            r_in = r_out
        lo = int(offset[h])
        pos[lo:lo + 16 * n] = np.concatenate(parts)
        vel[lo:lo + 16 * n] = rng.standard_normal((16 * n, 3)) * sigma_v
        radius[h] = 1.01 * r_in
    f = np.float32
    return Population(name=f"shell_profile_{'rise' if rise else 'fall'}", coord_type=COORD_F32_REL,
                      x=pos[:, 0].astype(f), y=pos[:, 1].astype(f), z=pos[:, 2].astype(f),
                      vx=vel[:, 0].astype(f), vy=vel[:, 1].astype(f), vz=vel[:, 2].astype(f),
                      m=None, m0=m0, box=0.0, centre=np.zeros((n_h, 3)), radius=radius, offset=offset,
                      count=counts, r200=np.zeros(n_h), conc=np.zeros(n_h))


def with_gas(pop, frac=0.3, u_max=5e4, seed=SEED_BASE + 7):
    """A copy of pop in which a random fraction of the particles are gas with
    a specific thermal energy uniform on [0, u_max) (km/s)^2 (the others 0),
    stored in the coordinates' precision."""
    rng = np.random.default_rng(seed)
    n = pop.n_particles
    gas = rng.uniform(0.0, 1.0, n) < frac
    u = np.where(gas, rng.uniform(0.0, u_max, n), 0.0).astype(pop.x.dtype)
    return dataclasses.replace(pop, u_th=u, name=pop.name + f"_gas{int(frac * 100)}")


def serving_stream(seed=SEED_BASE + 5, n_requests=50_000, rate_hz=10_000.0,
                   large_frac=0.05):
    """Poisson arrival times and per-request particle counts: 95 % from the
    power law on [100, 1e4), 5 % from [1e4, 1e5]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    big = rng.uniform(0.0, 1.0, n_requests) < large_frac
    counts = np.where(big, powerlaw_counts(rng, n_requests, 10_000, 100_000),
                      powerlaw_counts(rng, n_requests, 100, 9_999))
    return t, counts


WORKLOADS = {
    "single": single_halo,
    "batch": halo_batch,
    "tail": large_tail,
    "sweep": precision_sweep,
}

"""Plain FP64 CPU oracle of AHF's per-halo unbinding stage.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code with the CUDA path;
the only thing both sides consume is the seeded input generator, which holds
none of the method's arithmetic.

What it computes (Knollmann & Knebe 2009, "AHF: Amiga's Halo Finder"):

* Particle collection (Sect. 2.1): a halo's initial particle set is the
  sphere of a given radius around its centre.  Coordinates are recentred in
  FP64, with the minimum image in a periodic box (the paper's shift test in
  Sect. 3.2 relies on periodicity).
* Unbinding (Appendix A): the escape velocity is v_esc = sqrt(2|phi|); phi
  follows from integrating Poisson's equation for a spherical mass
  distribution, phi(r) = G int_0^r M(<r')/r'^2 dr' + phi_0, with phi_0 fixed by
  phi(infinity) = 0 for a halo truncated at its outer edge.  For the step
  function M(<r) of a particle list sorted by radius this integral is exact:

      phi_i = -G [ M(<r_i) / r_i + sum_{j >= i} m_j / r_j ]

  (integration by parts; the truncation radius drops out as long as it lies
  at or beyond the outermost particle).  Unbound particles are removed, phi_0
  and phi are re-evaluated for the new list, and the loop repeats until no
  particle is removed (Appendix A, last paragraph; Sect. 2.1).
* Virial radius (Sect. 2.1): mean enclosed density = Delta * rho_b, so
  M_vir = 4 pi rho_b Delta r_vir^3 / 3.

Readings where the paper is silent:

1. Bulk velocity: mass-weighted mean velocity of the current set, recomputed
   every iteration; the escape test uses u = v - v_bulk + H d (Hubble flow).
2. Removal: all unbound particles of an iteration are removed at once.
3. Truncation: at the current set's outermost particle.
4. Strict test: a particle is unbound iff |u|^2 > 2|phi|.
5. r = 0: with r_soft = 0 terms whose max(r_i, r_j) is 0 are dropped;
   r_soft > 0 replaces every radius r by max(r, r_soft).
6. r_vir is the first outward crossing: the first k (in the sorted final set,
   M_k the inclusive mass) with M_k < Delta rho (4 pi/3) r_{k+1}^3, with
   r_{N+1} = infinity, and r_vir = (3 M_k / (4 pi Delta rho))^(1/3).

Integral properties (Sect. 3.1, Sect. 3.2): the spin parameter and the
energies of the material within r_vir, the rotation curve's peak, and the
cross-identification of two catalogues by xi = N_shared^2 / (N_1 N_2); the
readings are in halo_properties and match_catalogs.

Pins: see tests/test_oracle_pins.py (brute force, Appendix A's integral
evaluated literally, analytic uniform-sphere and truncated-NFW potentials,
idempotence, the virial identity, invariances, special cases).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Per-halo status bits (mirrors the values documented in the C header; the
# numbers are part of the interface, not shared code).
OK = 0
NOT_CONVERGED = 1
EMPTY = 2
RVIR_BEYOND_EDGE = 4
RVIR_NONE = 8
RISE_EDGE = 16          # the extent is the rise of the density profile (variant)


@dataclasses.dataclass
class Params:
    G: float = 4.3009e-6
    H: float = 0.1
    delta_rho: float = 200.0 * 3.0 * 0.1 * 0.1 / (8.0 * math.pi * 4.3009e-6)
    r_soft: float = 0.0
    box: float = 0.0
    max_iter: int = 100
    band: float = 1e-5
    vbulk_initial: bool = False   # variant: v_bulk of the initial set in every iteration
    retruncate: bool = False      # variant: unbind again within r_vir (second pass)
    rise_edge: bool = False       # variant: extent at the rise of the density profile


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def recentre(x, y, z, centre, box):
    """d = x - c in FP64 (inputs promoted exactly), minimum image if box > 0."""
    d = np.stack([_f64(x) - centre[0], _f64(y) - centre[1], _f64(z) - centre[2]], axis=1)
    if box > 0.0:
        half = 0.5 * box
        d = np.where(d > half, d - box, d)
        d = np.where(d < -half, d + box, d)
    return d


def gas_energy(pop, h, member_idx=None):
    """The candidates' specific thermal energies (FP64), or None without gas."""
    if getattr(pop, "u_th", None) is None:
        return None
    lo = int(pop.offset[h])
    hi = lo + int(pop.count[h])
    pidx = np.arange(lo, hi, dtype=np.int64) if member_idx is None else np.asarray(member_idx[lo:hi], np.int64)
    return _f64(pop.u_th[pidx])


def gather_sphere(pop, h, member_idx=None):
    """Candidates of halo h and their recentred phase-space coordinates.

    Returns (pidx, d, v, m, inside): particle indices of the candidate slice,
    FP64 offsets from the centre, FP64 velocities, FP64 masses and the mask of
    candidates inside the gather sphere |d| <= R (Sect. 2.1)."""
    lo = int(pop.offset[h])
    hi = lo + int(pop.count[h])
    pidx = np.arange(lo, hi, dtype=np.int64) if member_idx is None else np.asarray(member_idx[lo:hi], np.int64)
    d = recentre(pop.x[pidx], pop.y[pidx], pop.z[pidx], pop.centre[h], pop.box)
    v = np.stack([_f64(pop.vx[pidx]), _f64(pop.vy[pidx]), _f64(pop.vz[pidx])], axis=1)
    m = np.full(pidx.shape[0], float(pop.m0)) if pop.m is None else _f64(pop.m[pidx])
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    R = float(pop.radius[h])
    inside = r2 <= R * R
    return pidx, d, v, m, inside


def potential_sorted(r, m, G, r_soft=0.0):
    """phi of particles sorted by radius (Appendix A, Eq. for phi and phi_0).

    M(<r_i) is the sequential FP64 sum of the masses before i; the outer sum
    is the sequential FP64 sum of m_j / r_j from the outermost particle in."""
    rr = np.maximum(r, r_soft)
    m_inner = np.concatenate([[0.0], np.cumsum(m)[:-1]])
    with np.errstate(divide="ignore", invalid="ignore"):
        mr = np.where(rr > 0.0, m / rr, 0.0)
        inner = np.where(rr > 0.0, m_inner / rr, 0.0)
    outer = np.cumsum(mr[::-1])[::-1]
    return -G * (inner + outer)


def potential_bruteforce(r, m, G, r_soft=0.0):
    """O(N^2) phi_i = -G sum_j m_j / max(r_i, r_j), zero-radius pairs dropped."""
    rr = np.maximum(_f64(r), r_soft)
    mx = np.maximum(rr[:, None], rr[None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(mx > 0.0, m[None, :] / mx, 0.0)
    return -G * t.sum(axis=1)


def virial(r, m, delta_rho):
    """First outward crossing of the mean enclosed density through delta_rho.

    r, m: the final set sorted by radius.  Returns (r_vir, m_vir, k, status)
    with k the 0-based index of the last particle inside r_vir."""
    n = r.shape[0]
    if n == 0:
        return 0.0, 0.0, -1, EMPTY
    mk = np.cumsum(m)
    r_next = np.concatenate([r[1:], [np.inf]])
    crit = delta_rho * (4.0 * math.pi / 3.0) * r_next ** 3
    k = int(np.argmax(mk < crit))          # first True; the last entry is always True
    m_vir = float(mk[k])
    r_vir = (3.0 * m_vir / (4.0 * math.pi * delta_rho)) ** (1.0 / 3.0)
    status = OK
    if k == n - 1:
        status |= RVIR_BEYOND_EDGE
    if m_vir < delta_rho * (4.0 * math.pi / 3.0) * r[k] ** 3:
        # the mean density never reaches delta_rho around any particle
        status |= RVIR_NONE
        return 0.0, 0.0, -1, status
    return r_vir, m_vir, k, status


RISE_SHELLS = 16        # equal-count shells of the bound set
RISE_MIN_N = 64         # fewer members: no density-profile edge


def rise_edge(r, m):
    """Edge of a halo whose mean overdensity never drops below the threshold:
    the rise of the density profile (Sect. 2.1, the truncation of subhaloes).

    The bound set, sorted by radius, is cut into RISE_SHELLS shells of equal
    particle count (shell s ends with particle b_s = (s+1) n / RISE_SHELLS - 1);
    the density of shell s is its mass over the volume between the radii of
    particles b_{s-1} and b_s.  Among the shells of the outer half (s >=
    RISE_SHELLS / 2) the first one of least density is the edge if a shell
    beyond it is denser; the halo then ends with its last particle.
    Returns that particle's index, or None (no rise, or too few members)."""
    n = r.shape[0]
    if n < RISE_MIN_N:
        return None
    b = [(s + 1) * n // RISE_SHELLS - 1 for s in range(RISE_SHELLS)]
    mk = np.cumsum(m)
    rho = {}
    for s in range(RISE_SHELLS // 2, RISE_SHELLS):
        lo, hi = b[s - 1], b[s]
        vol = 4.0 * math.pi / 3.0 * (float(r[hi]) ** 3 - float(r[lo]) ** 3)
        rho[s] = (mk[hi] - mk[lo]) / vol if vol > 0.0 else math.inf
    smin = min(rho, key=lambda s: (rho[s], s))
    if any(rho[s] > rho[smin] for s in rho if s > smin):
        return b[smin]
    return None


def unbind_halo(d, v, m, inside, params: Params, forced=None, u_th=None):
    """Iterative unbinding of one halo (Appendix A; Sect. 2.1).

    d, v, m: FP64 candidates (in candidate order); inside: gather-sphere mask.
    u_th: optional per-candidate specific thermal energy (gas particles): the
    escape test becomes |u|^2 + 2 u_th > 2|phi| (Sect. 2.1: the thermal energy
    of SPH gas particles counts in the unbinding).
    forced: optional per-candidate removal iteration (0 = never) used only for
    particles whose escape margin |(|u|^2 - 2|phi|) / 2|phi|| is below
    params.band (replay of another implementation's in-band decisions).

    Returns a dict with the final set (candidate positions sorted by (r, pos)),
    phi of the final set, per-candidate removal iteration (-1 outside the
    sphere, 0 bound, t removed in iteration t) and the iteration statistics."""
    n_cand = d.shape[0]
    r = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2 + d[:, 2] ** 2)
    removed_iter = np.where(inside, 0, -1).astype(np.int64)
    alive = np.nonzero(inside)[0]
    n_member = int(alive.shape[0])
    n_iter = 0
    part_iter = 0
    n_band = 0
    status = OK
    converged = False
    phi = np.zeros(0)
    order = alive
    while alive.shape[0] > 0 and n_iter < params.max_iter:
        n_iter += 1
        part_iter += int(alive.shape[0])
        ma = m[alive]
        if n_iter == 1 or not params.vbulk_initial:
            vbulk = (ma[:, None] * v[alive]).sum(axis=0) / ma.sum()
        # integrate along the radially ordered list (ties by candidate position)
        order = alive[np.lexsort((alive, r[alive]))]
        phi = potential_sorted(r[order], m[order], params.G, params.r_soft)
        u = v[order] - vbulk[None, :] + params.H * d[order]
        u2 = (u * u).sum(axis=1)
        if u_th is not None:
            u2 = u2 + 2.0 * u_th[order]
        two_phi = 2.0 * np.abs(phi)
        unbound = u2 > two_phi
        with np.errstate(divide="ignore", invalid="ignore"):
            margin = np.where(two_phi > 0.0, np.abs(u2 - two_phi) / two_phi, np.inf)
        in_band = margin < params.band
        n_band += int(in_band.sum())
        if forced is not None:
            fz = np.asarray(forced)[order] == n_iter
            unbound = np.where(in_band, fz, unbound)
        if not unbound.any():
            converged = True
            break
        removed_iter[order[unbound]] = n_iter
        alive = order[~unbound]
    if alive.shape[0] == 0:
        status |= EMPTY
        order = alive
        phi = np.zeros(0)
    elif not converged:
        status |= NOT_CONVERGED
        order = alive[np.lexsort((alive, r[alive]))]
        phi = potential_sorted(r[order], m[order], params.G, params.r_soft)
    if order.shape[0] > 0:
        mo = m[order]
        vbulk = (mo[:, None] * v[order]).sum(axis=0) / mo.sum()
        r_vir, m_vir, k_vir, vst = virial(r[order], mo, params.delta_rho)
        status |= vst
        if params.rise_edge and (vst & RVIR_BEYOND_EDGE) and not (vst & RVIR_NONE):
            k = rise_edge(r[order], mo)
            if k is not None:
                # the subhalo ends at the least dense shell before the rise
                k_vir, r_vir, m_vir = k, float(r[order][k]), float(np.cumsum(mo)[k])
                status |= RISE_EDGE
    else:
        vbulk = np.zeros(3)
        r_vir, m_vir, k_vir = 0.0, 0.0, -1
    return dict(order=order, phi=phi, r=r[order] if order.shape[0] else np.zeros(0),
                m=m[order] if order.shape[0] else np.zeros(0),
                removed_iter=removed_iter, n_member=n_member, n_iter=n_iter,
                part_iter=part_iter, n_band=n_band, status=status, vbulk=vbulk,
                r_vir=r_vir, m_vir=m_vir, k_vir=k_vir)


def retruncate_halo(o1, d, v, m, params: Params, u_th=None):
    """Variant: Appendix A truncates the potential at r_vir; after the
    unbinding converges, the bound particles within r_vir (all of them when
    there is no r_vir) are unbound again as a new halo.  The result is the
    second pass's, with the first pass's per-candidate removal iterations
    (candidates the second pass drops are visible only in the bound list)."""
    cand = o1["order"]
    if cand.shape[0] == 0:
        return o1
    inside = np.ones(cand.shape[0], dtype=bool)
    if o1["r_vir"] > 0.0:
        dc = d[cand]
        r2 = dc[:, 0] * dc[:, 0] + dc[:, 1] * dc[:, 1] + dc[:, 2] * dc[:, 2]
        inside = r2 <= o1["r_vir"] * o1["r_vir"]       # the gather sphere's test, radius r_vir
    o2 = unbind_halo(d[cand], v[cand], m[cand], inside, params, None, None if u_th is None else u_th[cand])
    o2["order"] = cand[o2["order"]]
    o2["removed_iter"] = o1["removed_iter"]
    return o2


def profile(r_sorted, m_sorted, r_vir, n_bins, r_min_frac, G):
    """Log-radial profile of a bound set (Sect. 2.1: radially binned output).

    Bin b covers (e_b, e_{b+1}] with e_b = r_out * f^(1 - b/n), r_out = r_vir
    (or the outermost particle when r_vir is 0).  Columns: particle count,
    mass within e_{b+1}, density of the bin's shell, circular velocity
    sqrt(G M(<=e_{b+1}) / e_{b+1})."""
    out = np.zeros((n_bins, 4))
    if r_sorted.shape[0] == 0:
        return out
    r_out = r_vir if r_vir > 0.0 else float(r_sorted[-1])
    edges = r_out * r_min_frac ** (1.0 - np.arange(n_bins + 1) / n_bins)
    edges[-1] = r_out
    for b in range(n_bins):
        lo, hi = edges[b], edges[b + 1]
        sel = (r_sorted > lo) & (r_sorted <= hi)
        mass_in = float(m_sorted[r_sorted <= hi].sum())
        out[b, 0] = float(sel.sum())
        out[b, 1] = mass_in
        out[b, 2] = float(m_sorted[sel].sum()) / (4.0 * math.pi / 3.0 * (hi ** 3 - lo ** 3))
        out[b, 3] = math.sqrt(G * mass_in / hi)
    return out


def halo_properties(d, v, m, phi, k_vir, params: Params):
    """Integral properties of a halo's bound set (Sect. 3.1's spin parameter,
    lambda = J sqrt|E| / (G M^(5/2)) after Peebles 1969; the rotation curve's
    peak).

    d, v, m: offsets from the centre, velocities and masses of the bound set
    in radial order (FP64); phi: its potential from the final iteration;
    k_vir: index of the last particle inside r_vir (-1: no r_vir).

    The material within r_vir is the first k_vir + 1 particles (the whole set
    when there is no r_vir).  Over it: M = sum m; v_bar = sum m v / M;
    u = v - v_bar + H d (the unbinding's frame); J = sum m d x u;
    K = sum m |u|^2 / 2; U = sum m phi / 2; E = K + U; and the circular
    velocity v_c(r_i) = sqrt(G M(<= r_i) / r_i), whose maximum is v_max at r_max
    (the first radius reaching it).  Returns a dict of those values and n."""
    d, v, m, phi = _f64(d), _f64(v), _f64(m), _f64(phi)
    n = d.shape[0] if k_vir < 0 else k_vir + 1
    out = dict(n=int(n), M=0.0, J=np.zeros(3), K=0.0, U=0.0, E=0.0, lam=0.0, v_max=0.0, r_max=0.0)
    if n == 0:
        return out
    d, v, m, phi = d[:n], v[:n], m[:n], phi[:n]
    M = float(m.sum())
    vbar = (m[:, None] * v).sum(axis=0) / M
    u = v - vbar[None, :] + params.H * d
    J = (m[:, None] * np.cross(d, u)).sum(axis=0)
    K = 0.5 * float((m * (u * u).sum(axis=1)).sum())
    U = 0.5 * float((m * phi).sum())
    E = K + U
    lam = float(np.sqrt((J * J).sum()) * math.sqrt(abs(E)) / (params.G * M ** 2.5))
    r = np.sqrt((d * d).sum(axis=1))
    m_in = np.cumsum(m)
    with np.errstate(divide="ignore", invalid="ignore"):
        vc = np.where(r > 0.0, np.sqrt(params.G * m_in / r), 0.0)
    i = int(np.argmax(vc))
    out.update(M=M, J=J, K=K, U=U, E=E, lam=lam, v_max=float(vc[i]), r_max=float(r[i]))
    return out


def match_catalogs(lists_a, lists_b):
    """Cross-identification of two halo catalogues (Sect. 3.2): for every halo
    of the first, the halo of the second maximising xi = N_shared^2 / (N_1 N_2),
    N_shared the particles the two have in common and N_1, N_2 their sizes.
    lists_a, lists_b: sequences of particle-id arrays (one per halo).  Returns
    (best, shared, xi) arrays over the first catalogue; best = -1 and xi = 0
    when a halo shares no particle (ties: the lower index of the second
    catalogue)."""
    owner = {}
    for b, ids in enumerate(lists_b):
        for i in np.asarray(ids).tolist():
            owner.setdefault(i, []).append(b)
    n_a = len(lists_a)
    best = np.full(n_a, -1, dtype=np.int64)
    shared = np.zeros(n_a, dtype=np.int64)
    xi = np.zeros(n_a)
    for a, ids in enumerate(lists_a):
        count = {}
        for i in np.asarray(ids).tolist():
            for b in owner.get(i, ()):
                count[b] = count.get(b, 0) + 1
        n1 = len(ids)
        for b in sorted(count):
            x = count[b] ** 2 / (n1 * len(lists_b[b]))
            if x > xi[a]:
                best[a], shared[a], xi[a] = b, count[b], x
    return best, shared, xi


def unbind_population(pop, params: Params, halos=None, member_idx=None,
                      forced=None, n_bins=0, r_min_frac=0.01, properties=False):
    """Run the oracle over haloes of a population (all of them by default).

    forced: optional per-candidate-slot removal iterations (flat, aligned
    with the candidate slices) for the in-band replay.
    Returns {h: result dict} with particle indices in 'bound_idx'."""
    res = {}
    hs = range(pop.n_halos) if halos is None else halos
    p = dataclasses.replace(params, box=pop.box)
    for h in hs:
        pidx, d, v, m, inside = gather_sphere(pop, h, member_idx)
        lo = int(pop.offset[h])
        fz = None if forced is None else np.asarray(forced[lo:lo + pidx.shape[0]])
        uth = gas_energy(pop, h, member_idx)
        o = unbind_halo(d, v, m, inside, p, fz, uth)
        if p.retruncate:
            o = retruncate_halo(o, d, v, m, p, uth)
        o["bound_idx"] = pidx[o["order"]]
        if n_bins > 0:
            o["profile"] = profile(o["r"], m[o["order"]], o["r_vir"], n_bins, r_min_frac, p.G)
        if properties:
            o["props"] = halo_properties(d[o["order"]], v[o["order"]], m[o["order"]], o["phi"], o["k_vir"], p)
        res[h] = o
    return res


def halo_depths(parent):
    """Depth of every halo in the forest given by parent (-1: none); raises
    ValueError on an index out of range or a cycle."""
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.shape[0]
    depth = np.full(n, -1, dtype=np.int64)
    for h in range(n):
        chain, k = [], h
        while k >= 0 and depth[k] < 0:
            if k in chain or parent[k] >= n or parent[k] < -1:
                raise ValueError("parent indices must form a forest")
            chain.append(k)
            k = int(parent[k])
        base = -1 if k < 0 else int(depth[k])
        for i, c in enumerate(reversed(chain)):
            depth[c] = base + 1 + i
    return depth


def unbind_hierarchy(pop, params: Params, parent, member_idx=None, forced=None):
    """Hosts and subhaloes in dependency order (Sect. 2.1): subhaloes are
    unbound before their hosts, and a host's candidates lose the particles
    that any of its descendants bound (the paper's option of not including
    subhaloes in their hosts; particles a subhalo does not bind stay the
    host's candidates).  Haloes are taken deepest level first; within a level
    independently, after which each particle's owner becomes the halo of that
    level that bound it (the highest index if several did).  A candidate is
    dropped from halo h when its owner descends from h.  Returns {h: result}
    as unbind_population does (excluded candidates count as outside the
    sphere: removed_iter -1).  forced: as for unbind_population."""
    parent = np.asarray(parent, dtype=np.int64)
    depth = halo_depths(parent)
    p = dataclasses.replace(params, box=pop.box)
    owner = {}

    def descends(t, h):
        while t >= 0:
            t = int(parent[t])
            if t == h:
                return True
        return False
    res = {}
    for d in sorted(set(depth.tolist()), reverse=True):
        level = [h for h in range(len(parent)) if depth[h] == d]
        for h in level:
            pidx, dd, v, m, inside = gather_sphere(pop, h, member_idx)
            keep = np.array([not descends(owner.get(int(q), -1), h) for q in pidx], dtype=bool)
            lo = int(pop.offset[h])
            fz = None if forced is None else np.asarray(forced[lo:lo + pidx.shape[0]])
            o = unbind_halo(dd, v, m, inside & keep, p, fz, gas_energy(pop, h, member_idx))
            o["bound_idx"] = pidx[o["order"]]
            res[h] = o
        for h in level:                      # ascending: the highest index of a level wins
            for q in res[h]["bound_idx"].tolist():
                owner[q] = h
    return res


def _worker(args):
    import time
    pop, params, n_bins, r_min_frac = args
    t0 = time.perf_counter()
    out = unbind_population(pop, params, n_bins=n_bins, r_min_frac=r_min_frac)
    dt = time.perf_counter() - t0
    return [(o["n_iter"], o["part_iter"], o["order"].shape[0]) for _, o in sorted(out.items())], dt


def unbind_population_parallel(pop, params: Params, halos, n_workers, n_bins=0, r_min_frac=0.01, chunks=None):
    """The oracle over haloes spread across n_workers spawned processes
    (the i-th listed halo goes to worker i % n_workers, unless `chunks`
    gives each worker's haloes).  Returns
    ({h: (n_iter, part_iter, n_bound)}, the longest worker's compute time in
    seconds, process start-up excluded).  Used only to time the oracle as a
    CPU baseline; the arithmetic is unbind_population's."""
    import multiprocessing as mp
    halos = list(halos)
    if chunks is None:
        chunks = [halos[i::n_workers] for i in range(n_workers)]
    chunks = [list(c) for c in chunks if len(c)]
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(len(chunks)) as pool:
        parts = pool.map(_worker, [(_subset(pop, c), params, n_bins, r_min_frac) for c in chunks])
    for c, (part, _) in zip(chunks, parts):
        for h, stats in zip(c, part):
            res[h] = stats
    return res, max(dt for _, dt in parts)


def _subset(pop, halos):
    """A population holding only the given haloes (renumbered 0..k-1)."""
    import copy
    halos = list(halos)
    idx = np.concatenate([np.arange(pop.offset[h], pop.offset[h] + pop.count[h]) for h in halos])
    sub = copy.copy(pop)
    for a in ("x", "y", "z", "vx", "vy", "vz"):
        setattr(sub, a, getattr(pop, a)[idx])
    sub.m = None if pop.m is None else pop.m[idx]
    if getattr(pop, "u_th", None) is not None:
        sub.u_th = pop.u_th[idx]
    cnt = pop.count[halos]
    sub.count = cnt.copy()
    sub.offset = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
    for a in ("centre", "radius", "r200", "conc"):
        setattr(sub, a, getattr(pop, a)[halos])
    return sub

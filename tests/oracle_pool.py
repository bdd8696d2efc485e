"""Oracle comparisons spread over the host cores.

Large parity cases (1e5 haloes, 1e8 particles) take the single-core oracle
minutes.  Here the population and the GPU outputs are copied once into
shared memory; spawned worker processes (spawn: the parent has a CUDA
context, which a forked child must not inherit) attach to the same pages and
each runs tests.parity.compare on a share of the haloes.  The arithmetic is
compare's and the oracle's; this module only moves data.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import types
from multiprocessing import shared_memory

import numpy as np

_POP_ARRAYS = ("x", "y", "z", "vx", "vy", "vz", "m", "u_th", "centre", "radius", "offset", "count")


class _Shared:
    def __init__(self):
        self.blocks = []
        self.spec = {}

    def put(self, name, arr):
        if arr is None:
            self.spec[name] = None
            return
        arr = np.ascontiguousarray(arr)
        shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
        np.ndarray(arr.shape, arr.dtype, buffer=shm.buf)[...] = arr
        self.blocks.append(shm)
        self.spec[name] = (shm.name, arr.shape, arr.dtype)

    def close(self):
        for b in self.blocks:
            b.close()
            b.unlink()


def _attach(spec):
    out, handles = {}, []
    for name, s in spec.items():
        if s is None:
            out[name] = None
            continue
        shm = shared_memory.SharedMemory(name=s[0])
        handles.append(shm)
        out[name] = np.ndarray(s[1], s[2], buffer=shm.buf)
    return out, handles


def _work(args):
    spec, meta, params, halos, kw = args
    from tests.parity import compare
    a, handles = _attach(spec)
    try:
        pop = types.SimpleNamespace(**meta, **{k: a[k] for k in _POP_ARRAYS})
        return compare(pop, params, a["res"], a["bound_idx"], a["phi"], a["removed_iter"], halos=halos, **kw)
    finally:
        del a
        for h in handles:
            h.close()


def compare_parallel(pop, params, res, bound_idx, phi, removed_iter, workers=None, **kw):
    """tests.parity.compare over every halo of `pop`, on `workers` spawned
    processes (default: the host's cores).  Returns the combined summary;
    raises the first worker's AssertionError."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    sh = _Shared()
    try:
        for k in _POP_ARRAYS:
            sh.put(k, getattr(pop, k, None))
        sh.put("res", res)
        sh.put("bound_idx", bound_idx)
        sh.put("phi", phi)
        sh.put("removed_iter", removed_iter)
        meta = {"coord_type": pop.coord_type, "m0": pop.m0, "box": pop.box, "name": pop.name,
                "n_halos": pop.n_halos}
        prm = types.SimpleNamespace(**{f: getattr(params, f) for f in
                                       ("G", "H", "delta_rho", "r_soft", "box", "band", "max_iter",
                                        "precision", "variant")})
        # largest first, dealt out in 4 * workers shares of similar candidate counts
        order = np.argsort(-np.asarray(pop.count), kind="stable")
        n_share = 4 * workers
        shares = [[] for _ in range(n_share)]
        load = np.zeros(n_share)
        for h in order:
            j = int(np.argmin(load))
            shares[j].append(int(h))
            load[j] += float(pop.count[h])
        jobs = [(sh.spec, meta, prm, sorted(s), kw) for s in shares if s]
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            parts = pool.map(_work, jobs, chunksize=1)
    finally:
        sh.close()
    out = {"worst_phi_rel": 0.0, "worst_vir_rel": 0.0, "n_band": 0, "worst_order_inversion": 0.0, "halos": 0}
    for p in parts:
        out["worst_phi_rel"] = max(out["worst_phi_rel"], float(p["worst_phi_rel"]))
        out["worst_vir_rel"] = max(out["worst_vir_rel"], float(p["worst_vir_rel"]))
        out["worst_order_inversion"] = max(out["worst_order_inversion"], float(p["worst_order_inversion"]))
        out["n_band"] += int(p["n_band"])
        out["halos"] += int(p["halos"])
    return out

"""Thin Python binding of libahfgpu (argument marshalling only).

Every step of the unbinding stage runs in the library's CUDA kernels; this
module only turns torch tensors and numpy descriptors into the C structs of
include/ahf.h and back.  PyTorch provides device memory and streams.  There
is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libahfgpu.so")

# status / codes (values from include/ahf.h)
OK, PENDING = 0, 1
ERR_INVALID, ERR_NOMEM, ERR_TIMEOUT, ERR_CUDA, ERR_FULL, ERR_NOT_FOUND = -1, -2, -3, -4, -5, -6
HALO_OK, HALO_NOT_CONVERGED, HALO_EMPTY, HALO_RVIR_BEYOND_EDGE, HALO_RVIR_NONE = 0, 1, 2, 4, 8
HALO_RISE_EDGE = 16
COORD_F64, COORD_F32_REL, COORD_F32_BOX = 0, 1, 2
PREC_MIXED, PREC_FP64 = 0, 1
VAR_VBULK_INITIAL, VAR_RETRUNCATE, VAR_RISE_EDGE = 1, 2, 4
OPT_ONCHIP_MAX, OPT_WAIT_LIMIT, OPT_TIMING, OPT_HOST_DIRECT, OPT_GRAPHS, OPT_TRACE, OPT_SERIAL = 1, 2, 3, 4, 5, 6, 7
OPT_PROMOTE = 8
OPT_PASS_CHUNK = 9
OPT_WORKSPACE_CAP = 10
OPT_CLASS_CUT = 16                 # + variant (0..7)
TRACE_FIELDS = 8
N_PHASES = 12
PHASE_NAMES = ("warp_512", "cta_1k", "cta_4k", "cta_8k", "cluster2_16k", "cluster4_32k", "cluster8_64k",
               "cluster16_128k", "grid_gather_sort", "grid_iterate", "grid_finish", "profile")
VARIANT_CAPS = (512, 1024, 4096, 8192, 2 * 8192, 4 * 8192, 8 * 8192, 16 * 8192)

HALO_DTYPE = np.dtype([("cx", "<f8"), ("cy", "<f8"), ("cz", "<f8"), ("radius", "<f8"),
                       ("offset", "<i8"), ("count", "<i8")])
RESULT_DTYPE = np.dtype([("n_bound", "<i8"), ("n_member", "<i8"), ("part_iter", "<i8"), ("n_band", "<i8"),
                         ("k_vir", "<i8"), ("n_iter", "<i4"), ("status", "<i4"), ("m_vir", "<f8"),
                         ("r_vir", "<f8"), ("vbulk", "<f8", (3,))])
assert HALO_DTYPE.itemsize == 48 and RESULT_DTYPE.itemsize == 88

# every symbol include/ahf.h declares
EXPORTS = ("ahf_version", "ahf_last_error", "ahf_create", "ahf_destroy", "ahf_unbind_batch",
           "ahf_unbind_batch_host", "ahf_unbind_plain", "ahf_profile_batch", "ahf_set_option",
           "ahf_get_option", "ahf_sync", "ahf_get_stats", "ahf_unbind_batch_static", "ahf_unbind_profile_batch",
           "ahf_serve_create", "ahf_serve_submit", "ahf_serve_poll", "ahf_serve_stats", "ahf_serve_counters",
           "ahf_serve_reset_stats", "ahf_serve_destroy", "ahf_get_trace", "ahf_halo_properties",
           "ahf_match_catalogs", "ahf_unbind_hierarchy", "ahf_build_id")
PROP_FIELDS = 12
SERVE_MAX_COUNT = 131072
STATIC_MAX_HALOS, STATIC_MAX_COUNT = 32768, 8192


class AHFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libahfgpu error {code}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("H", ctypes.c_double), ("delta_rho", ctypes.c_double),
                ("r_soft", ctypes.c_double), ("box", ctypes.c_double), ("band", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _Particles(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("m", ctypes.c_void_p), ("m0", ctypes.c_double), ("n", ctypes.c_int64),
                ("coord_type", ctypes.c_int32), ("reserved", ctypes.c_int32), ("u_th", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("host_syncs", ctypes.c_int64),
                ("grid_iterations", ctypes.c_int64),
                ("phase_halos", ctypes.c_int64 * N_PHASES), ("phase_candidates", ctypes.c_int64 * N_PHASES),
                ("phase_ms", ctypes.c_double * N_PHASES), ("graph_launches", ctypes.c_int64),
                ("graph_captures", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libahfgpu.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built: run paper_0904_3662_gb300.build_lib.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.ahf_version.restype = ctypes.c_int
    lib.ahf_last_error.restype = ctypes.c_char_p
    lib.ahf_build_id.restype = ctypes.c_char_p
    lib.ahf_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.ahf_destroy.argtypes = [vp]
    sig = [vp, ctypes.POINTER(_Particles), vp, i64, vp, ctypes.POINTER(_Params), vp, vp, vp, vp, vp]
    for name in ("ahf_unbind_batch", "ahf_unbind_plain"):
        getattr(lib, name).argtypes = sig
    lib.ahf_unbind_batch_host.argtypes = sig[:-1] + [i32, ctypes.c_double, vp, vp]
    lib.ahf_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.ahf_unbind_batch_static.argtypes = sig[1:-1] + [vp, vp]
    lib.ahf_unbind_hierarchy.argtypes = sig[:4] + [vp] + sig[4:]
    lib.ahf_unbind_profile_batch.argtypes = sig[:-1] + [i32, ctypes.c_double, vp, vp]
    if hasattr(lib, "ahf_profile_batch"):
        lib.ahf_profile_batch.argtypes = [vp, ctypes.POINTER(_Particles), vp, i64, vp, ctypes.POINTER(_Params),
                                          vp, vp, i32, ctypes.c_double, vp, vp]
    lib.ahf_set_option.argtypes = [vp, ctypes.c_int, i64]
    lib.ahf_get_option.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64)]
    lib.ahf_sync.argtypes = [vp]
    lib.ahf_get_trace.argtypes = [vp, vp, i64]
    lib.ahf_halo_properties.argtypes = [vp, ctypes.POINTER(_Particles), vp, i64, vp, ctypes.POINTER(_Params),
                                        vp, vp, vp, vp, vp]
    lib.ahf_match_catalogs.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.ahf_serve_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_Params),
                                     i32, ctypes.c_double]
    lib.ahf_serve_submit.argtypes = [vp, ctypes.POINTER(_Particles), vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.ahf_serve_poll.argtypes = [vp, ctypes.c_uint64, vp, vp, i64]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.ahf_serve_stats.argtypes = [vp, dp, dp, dp]
    ip = ctypes.POINTER(i64)
    lib.ahf_serve_counters.argtypes = [vp, ip, ip, ip, ip]
    lib.ahf_serve_reset_stats.argtypes = [vp]
    lib.ahf_serve_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _check(rc):
    if rc < 0:
        raise AHFError(rc, _lib.ahf_last_error().decode())
    return rc


@dataclasses.dataclass
class Params:
    """Mirror of ahf_params (defaults: kpc/h, km/s, Msun/h; Delta = 200 rho_crit)."""
    G: float = 4.3009e-6
    H: float = 0.1
    delta_rho: float = 200.0 * 3.0 * 0.1 * 0.1 / (8.0 * math.pi * 4.3009e-6)
    r_soft: float = 0.0
    box: float = 0.0
    band: float = 1e-5
    max_iter: int = 100
    precision: int = PREC_MIXED
    variant: int = 0

    def c(self):
        return _Params(self.G, self.H, self.delta_rho, self.r_soft, self.box, self.band,
                       self.max_iter, self.precision, self.variant, 0)


def halo_array(centre, radius, offset, count):
    """Host halo descriptors as the C struct layout."""
    n = len(offset)
    h = np.zeros(n, dtype=HALO_DTYPE)
    centre = np.asarray(centre, dtype=np.float64).reshape(n, 3)
    h["cx"], h["cy"], h["cz"] = centre[:, 0], centre[:, 1], centre[:, 2]
    h["radius"] = np.asarray(radius, dtype=np.float64)
    h["offset"] = np.asarray(offset, dtype=np.int64)
    h["count"] = np.asarray(count, dtype=np.int64)
    return h


@dataclasses.dataclass
class Particles:
    """Particle store: torch tensors (device) or numpy arrays (host)."""
    x: object
    y: object
    z: object
    vx: object
    vy: object
    vz: object
    m: object = None
    m0: float = 0.0
    coord_type: int = COORD_F32_REL
    u_th: object = None       # gas: specific thermal energy per particle, or None

    @property
    def n(self):
        return int(self.x.shape[0])

    def c(self):
        def ptr(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                return a.ctypes.data
            return a.data_ptr()
        return _Particles(ptr(self.x), ptr(self.y), ptr(self.z), ptr(self.vx), ptr(self.vy), ptr(self.vz),
                          ptr(self.m), float(self.m0), self.n, int(self.coord_type), 0, ptr(self.u_th))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def n_slots_of(halos, n_particles, member_idx):
    if member_idx is None:
        return int(n_particles)
    return int((halos["offset"] + halos["count"]).max()) if len(halos) else 0


class Context:
    """An ahf_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self._p = ctypes.c_void_p()
        _check(self.lib.ahf_create(ctypes.byref(self._p), int(device)))
        self.device = device

    def close(self):
        if self._p:
            self.lib.ahf_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, opt, value):
        _check(self.lib.ahf_set_option(self._p, int(opt), int(value)))

    def get_option(self, opt):
        v = ctypes.c_int64()
        _check(self.lib.ahf_get_option(self._p, int(opt), ctypes.byref(v)))
        return v.value

    def sync(self):
        _check(self.lib.ahf_sync(self._p))

    def stats(self):
        st = _Stats()
        _check(self.lib.ahf_get_stats(self._p, ctypes.byref(st)))
        return {"launches": st.launches, "host_syncs": st.host_syncs, "grid_iterations": st.grid_iterations,
                "phase_halos": list(st.phase_halos), "phase_candidates": list(st.phase_candidates),
                "phase_ms": list(st.phase_ms), "graph_launches": st.graph_launches,
                "graph_captures": st.graph_captures}

    def halo_properties(self, parts: Particles, halos, params: Params, out, member_idx=None, stream=None):
        """ahf_halo_properties over the outputs `out` of an unbinding call:
        device double (n_halos, PROP_FIELDS)."""
        import torch
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        props = torch.empty((len(halos), PROP_FIELDS), dtype=torch.float64, device=torch.device("cuda", self.device))
        pc, prc = parts.c(), params.c()
        _check(self.lib.ahf_halo_properties(
            self._p, ctypes.byref(pc), halos.ctypes.data, len(halos),
            None if member_idx is None else member_idx.data_ptr(), ctypes.byref(prc), out["res"].data_ptr(),
            out["bound_idx"].data_ptr(), out["phi"].data_ptr(), props.data_ptr(), _stream_ptr(stream)))
        return props

    def match_catalogs(self, n_ids, ids_a, off_a, cnt_a, ids_b, off_b, cnt_b, stream=None):
        """ahf_match_catalogs on device int64 tensors: (best, shared, xi)."""
        import torch
        dev = torch.device("cuda", self.device)
        n_a, n_b = int(off_a.shape[0]), int(off_b.shape[0])
        best = torch.empty(max(n_a, 1), dtype=torch.int64, device=dev)
        shared = torch.empty(max(n_a, 1), dtype=torch.int64, device=dev)
        xi = torch.empty(max(n_a, 1), dtype=torch.float64, device=dev)
        _check(self.lib.ahf_match_catalogs(
            self._p, int(n_ids), ids_a.data_ptr(), off_a.data_ptr(), cnt_a.data_ptr(), n_a, ids_b.data_ptr(),
            off_b.data_ptr(), cnt_b.data_ptr(), n_b, best.data_ptr(), shared.data_ptr(), xi.data_ptr(),
            _stream_ptr(stream)))
        return best[:n_a], shared[:n_a], xi[:n_a]

    def trace(self, n_halos):
        """Per-halo trace of the last call made with OPT_TRACE on:
        (n_halos, TRACE_FIELDS) int64 (see ahf_get_trace)."""
        t = np.zeros((n_halos, TRACE_FIELDS), dtype=np.int64)
        _check(self.lib.ahf_get_trace(self._p, t.ctypes.data, int(n_halos)))
        return t

    def alloc_outputs(self, n_halos, n_slots, with_phi=True, with_removed=True, precision=PREC_MIXED):
        import torch
        dev = torch.device("cuda", self.device)
        out = {
            "res": torch.empty(n_halos * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev),
            "bound_idx": torch.empty(max(n_slots, 1), dtype=torch.int64, device=dev),
            "phi": None, "removed_iter": None,
        }
        if with_phi:
            out["phi"] = torch.empty(max(n_slots, 1), device=dev,
                                     dtype=torch.float64 if precision == PREC_FP64 else torch.float32)
        if with_removed:
            out["removed_iter"] = torch.empty(max(n_slots, 1), dtype=torch.int32, device=dev)
        return out

    def unbind_batch(self, parts: Particles, halos, params: Params, member_idx=None, out=None,
                     with_phi=True, with_removed=True, stream=None, plain=False):
        """Enqueue ahf_unbind_batch (or ahf_unbind_plain) on `stream`."""
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        n_slots = n_slots_of(halos, parts.n, member_idx)
        if out is None:
            out = self.alloc_outputs(len(halos), n_slots, with_phi, with_removed, params.precision)
        pc, prc = parts.c(), params.c()
        fn = self.lib.ahf_unbind_plain if plain else self.lib.ahf_unbind_batch
        _check(fn(self._p, ctypes.byref(pc), halos.ctypes.data, len(halos),
                  None if member_idx is None else member_idx.data_ptr(), ctypes.byref(prc),
                  out["res"].data_ptr(), out["bound_idx"].data_ptr(),
                  None if out["phi"] is None else out["phi"].data_ptr(),
                  None if out["removed_iter"] is None else out["removed_iter"].data_ptr(),
                  _stream_ptr(stream)))
        return out

    def unbind_hierarchy(self, parts: Particles, halos, parent, params: Params, member_idx=None, out=None,
                         with_phi=True, with_removed=True, stream=None):
        """ahf_unbind_hierarchy: hosts after their subhaloes, each host without
        the particles its descendants bound.  parent: host index per halo
        (-1 for none)."""
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        parent = np.ascontiguousarray(parent, dtype=np.int64)
        if parent.shape != (len(halos),):
            raise ValueError("parent needs one entry per halo")
        n_slots = n_slots_of(halos, parts.n, member_idx)
        if out is None:
            out = self.alloc_outputs(len(halos), n_slots, with_phi, with_removed, params.precision)
        pc, prc = parts.c(), params.c()
        _check(self.lib.ahf_unbind_hierarchy(
            self._p, ctypes.byref(pc), halos.ctypes.data, len(halos), parent.ctypes.data,
            None if member_idx is None else member_idx.data_ptr(), ctypes.byref(prc),
            out["res"].data_ptr(), out["bound_idx"].data_ptr(),
            None if out["phi"] is None else out["phi"].data_ptr(),
            None if out["removed_iter"] is None else out["removed_iter"].data_ptr(),
            _stream_ptr(stream)))
        return out

    def unbind_profile_batch(self, parts: Particles, halos, params: Params, n_bins=32, r_min_frac=0.01,
                             member_idx=None, out=None, prof=None, with_phi=True, with_removed=True, stream=None):
        """ahf_unbind_profile_batch: unbinding and profile rows in one call."""
        import torch
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        n_slots = n_slots_of(halos, parts.n, member_idx)
        if out is None:
            out = self.alloc_outputs(len(halos), n_slots, with_phi, with_removed, params.precision)
        if prof is None:
            prof = torch.empty((len(halos), n_bins, 4), dtype=torch.float64, device=torch.device("cuda", self.device))
        pc, prc = parts.c(), params.c()
        _check(self.lib.ahf_unbind_profile_batch(
            self._p, ctypes.byref(pc), halos.ctypes.data, len(halos),
            None if member_idx is None else member_idx.data_ptr(), ctypes.byref(prc),
            out["res"].data_ptr(), out["bound_idx"].data_ptr(),
            None if out["phi"] is None else out["phi"].data_ptr(),
            None if out["removed_iter"] is None else out["removed_iter"].data_ptr(),
            int(n_bins), float(r_min_frac), prof.data_ptr(), _stream_ptr(stream)))
        out["prof"] = prof
        return out

    def unbind_batch_host(self, parts: Particles, halos, params: Params, member_idx=None, out=None,
                          with_phi=True, with_removed=True, n_bins=0, r_min_frac=0.01, stream=None):
        """ahf_unbind_batch_host: numpy inputs and outputs in host memory
        (profile too when n_bins > 0)."""
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        n_slots = n_slots_of(halos, parts.n, member_idx)
        if out is None:
            out = {"res": np.zeros(len(halos), dtype=RESULT_DTYPE),
                   "bound_idx": np.zeros(max(n_slots, 1), dtype=np.int64),
                   "phi": np.zeros(max(n_slots, 1), dtype=np.float64 if params.precision == PREC_FP64
                                   else np.float32) if with_phi else None,
                   "removed_iter": np.zeros(max(n_slots, 1), dtype=np.int32) if with_removed else None,
                   "prof": np.zeros((len(halos), n_bins, 4)) if n_bins > 0 else None}
        pc, prc = parts.c(), params.c()

        def p(a):
            return None if a is None else a.ctypes.data
        _check(self.lib.ahf_unbind_batch_host(
            self._p, ctypes.byref(pc), halos.ctypes.data, len(halos),
            None if member_idx is None else member_idx.ctypes.data, ctypes.byref(prc),
            p(out["res"]), p(out["bound_idx"]), p(out["phi"]), p(out["removed_iter"]),
            int(n_bins), float(r_min_frac), p(out.get("prof")), _stream_ptr(stream)))
        return out

    def profile_batch(self, parts: Particles, halos, params: Params, res_dev, bound_idx, n_bins=32,
                      r_min_frac=0.01, member_idx=None, prof=None, stream=None):
        import torch
        halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
        if prof is None:
            prof = torch.empty((len(halos), n_bins, 4), dtype=torch.float64,
                               device=torch.device("cuda", self.device))
        pc, prc = parts.c(), params.c()
        _check(self.lib.ahf_profile_batch(self._p, ctypes.byref(pc), halos.ctypes.data, len(halos),
                                          None if member_idx is None else member_idx.data_ptr(),
                                          ctypes.byref(prc), res_dev.data_ptr(), bound_idx.data_ptr(),
                                          int(n_bins), float(r_min_frac), prof.data_ptr(), _stream_ptr(stream)))
        return prof


class Serve:
    """An ahf_serve instance: one-halo requests from host arrays, continuous
    batching on the device, non-blocking polls."""

    def __init__(self, params: Params, device: int = 0, hbm_cap_bytes: int = 1 << 30,
                 coord_type: int = COORD_F32_REL, m0: float = 0.0):
        self.lib = load_library()
        self._p = ctypes.c_void_p()
        self._prm = params.c()
        _check(self.lib.ahf_serve_create(ctypes.byref(self._p), int(device), int(hbm_cap_bytes),
                                         ctypes.byref(self._prm), int(coord_type), float(m0)))
        self._res = np.zeros(1, dtype=RESULT_DTYPE)
        self._bound = np.empty(SERVE_MAX_COUNT, dtype=np.int64)

    def close(self):
        if self._p:
            self.lib.ahf_serve_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def request(parts: Particles, halo):
        """Prepared arguments of one submission (numpy particle arrays and a
        one-element HALO_DTYPE array); keep the returned tuple alive until
        submit returns."""
        halo = np.ascontiguousarray(halo, dtype=HALO_DTYPE).reshape(1)
        return (parts.c(), halo, parts)

    def submit_prepared(self, req):
        """Return the request id, or None when the ring is full (AHF_ERR_FULL)."""
        rid = ctypes.c_uint64()
        rc = self.lib.ahf_serve_submit(self._p, ctypes.byref(req[0]), req[1].ctypes.data, ctypes.byref(rid))
        if rc == ERR_FULL:
            return None
        _check(rc)
        return rid.value

    def submit(self, parts: Particles, halo):
        return self.submit_prepared(self.request(parts, halo))

    def poll(self, req_id, cap=SERVE_MAX_COUNT):
        """None while pending, else (result record, bound indices)."""
        cap = max(1, min(int(cap), SERVE_MAX_COUNT))
        bound = self._bound
        rc = self.lib.ahf_serve_poll(self._p, int(req_id), self._res.ctypes.data, bound.ctypes.data, cap)
        if rc == PENDING:
            return None
        _check(rc)
        res = self._res[0].copy()
        return res, bound[:int(res["n_bound"])].copy()

    def stats(self):
        p50, p99, thr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.lib.ahf_serve_stats(self._p, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(thr)))
        c = [ctypes.c_int64() for _ in range(4)]
        _check(self.lib.ahf_serve_counters(self._p, *[ctypes.byref(x) for x in c]))
        return {"p50_us": p50.value, "p99_us": p99.value, "throughput": thr.value, "submitted": c[0].value,
                "completed": c[1].value, "rejected": c[2].value, "batches": c[3].value}

    def reset_stats(self):
        _check(self.lib.ahf_serve_reset_stats(self._p))


def results_to_numpy(res_tensor):
    """Decode a device result buffer into a numpy structured array."""
    raw = res_tensor.detach().cpu().numpy()
    return raw.view(RESULT_DTYPE)


def particles_from_population(pop, device="cuda"):
    """Device copies of a synthetic population's particle arrays."""
    import torch

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device)
    m = None if pop.m is None else t(pop.m)
    u = None if getattr(pop, "u_th", None) is None else t(pop.u_th)
    return Particles(t(pop.x), t(pop.y), t(pop.z), t(pop.vx), t(pop.vy), t(pop.vz), m, float(pop.m0),
                     int(pop.coord_type), u)


def halos_from_population(pop):
    return halo_array(pop.centre, pop.radius, pop.offset, pop.count)


def build_id() -> str:
    """The library's build id (a hash of its sources; tuning files are keyed by it)."""
    return load_library().ahf_build_id().decode()


def params_for(pop, **kw):
    return Params(box=float(pop.box), **kw)

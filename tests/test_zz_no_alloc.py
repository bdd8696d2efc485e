"""The allocation-free entry point, ahf_unbind_batch_static.

It exists for callers that cannot let a library allocate device memory:
applications whose GPU memory belongs to another allocator, and loops that
must not block in cudaMalloc / cudaFree.  Its scratch is one fixed array in
device memory shared by every call, so the checks below run two different
batches back to back and compare each with ahf_unbind_batch on the same
inputs (same kernels, so results must agree to the parity tolerance; they
are in fact expected to be identical).

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_0904_3662_gb300 import ahf, synth


def _call_static(parts, halos, prm, out, stream):
    lib = ahf.load_library()
    pc, prc = parts.c(), prm.c()
    rc = lib.ahf_unbind_batch_static(ctypes.byref(pc), halos.ctypes.data, len(halos), None, ctypes.byref(prc),
                                     out["res"].data_ptr(), out["bound_idx"].data_ptr(), out["phi"].data_ptr(),
                                     out["removed_iter"].data_ptr(), stream)
    return rc


def test_static_rejects_oversized_requests_without_a_gpu():
    from paper_0904_3662_gb300 import build_lib
    build_lib.build()
    lib = ahf.load_library()
    pop = synth.halo_batch(seed=21, n_halos=2, n_lo=100, n_hi=200)
    parts = ahf.Particles(pop.x, pop.y, pop.z, pop.vx, pop.vy, pop.vz, None, pop.m0, pop.coord_type)
    prm = ahf.params_for(pop)
    pc, prc = parts.c(), prm.c()
    big = np.zeros(ahf.STATIC_MAX_HALOS + 1, dtype=ahf.HALO_DTYPE)
    rc = lib.ahf_unbind_batch_static(ctypes.byref(pc), big.ctypes.data, len(big), None, ctypes.byref(prc),
                                     None, None, None, None, None)
    assert rc == ahf.ERR_INVALID
    assert b"AHF_STATIC_MAX_HALOS" in lib.ahf_last_error()
    one = ahf.halos_from_population(pop)
    one["count"][0] = ahf.STATIC_MAX_COUNT + 1
    dummy = np.zeros(16, dtype=np.int64)
    rc = lib.ahf_unbind_batch_static(ctypes.byref(pc), one.ctypes.data, len(one), None, ctypes.byref(prc),
                                     dummy.ctypes.data, dummy.ctypes.data, None, None, None)
    assert rc == ahf.ERR_INVALID
    assert b"AHF_STATIC_MAX_COUNT" in lib.ahf_last_error()


@pytest.mark.gpu
def test_static_matches_batch_entry_point_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_3662_gb300 import build_lib
    build_lib.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = ahf.Context(0)
    # two batches of different shapes, every halo within the on-chip class
    pops = [synth.halo_batch(seed=22, n_halos=40, n_lo=100, n_hi=7000),
            synth.halo_batch(seed=23, n_halos=17, n_lo=300, n_hi=7000, coord_type=synth.COORD_F64,
                             with_masses=True)]
    for pop in pops:
        assert pop.count.max() <= ahf.STATIC_MAX_COUNT
    refs, outs = [], []
    for pop in pops:
        parts = ahf.particles_from_population(pop)
        hal = ahf.halos_from_population(pop)
        prm = ahf.params_for(pop)
        ref = ctx.unbind_batch(parts, hal, prm, stream=stream)
        out = ctx.alloc_outputs(len(hal), pop.n_particles)
        refs.append((pop, parts, hal, prm, ref, out))
    torch.cuda.synchronize()
    # the two static calls back to back on one stream
    for pop, parts, hal, prm, ref, out in refs:
        assert _call_static(parts, hal, prm, out, stream.cuda_stream) == ahf.OK, ahf.load_library().ahf_last_error()
    torch.cuda.synchronize()
    for pop, parts, hal, prm, ref, out in refs:
        a = ahf.results_to_numpy(ref["res"])
        b = ahf.results_to_numpy(out["res"])
        for k in ("n_bound", "n_member", "part_iter", "n_iter", "status", "k_vir", "n_band"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        np.testing.assert_allclose(b["m_vir"], a["m_vir"], rtol=1e-5)
        np.testing.assert_allclose(b["r_vir"], a["r_vir"], rtol=1e-5)
        np.testing.assert_array_equal(ref["removed_iter"].cpu().numpy(), out["removed_iter"].cpu().numpy())
        bi_a, bi_b = ref["bound_idx"].cpu().numpy(), out["bound_idx"].cpu().numpy()
        ph_a, ph_b = ref["phi"].cpu().numpy(), out["phi"].cpu().numpy()
        for h in range(pop.n_halos):
            lo, nb = int(pop.offset[h]), int(a["n_bound"][h])
            np.testing.assert_array_equal(bi_a[lo:lo + nb], bi_b[lo:lo + nb])
            np.testing.assert_allclose(ph_b[lo:lo + nb], ph_a[lo:lo + nb], rtol=1e-5)

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


def _call_static(parts, halos, prm, out, stream, member_idx=None, error_out=None):
    lib = ahf.load_library()
    pc, prc = parts.c(), prm.c()
    rc = lib.ahf_unbind_batch_static(ctypes.byref(pc), halos.ctypes.data, len(halos),
                                     None if member_idx is None else member_idx.data_ptr(), ctypes.byref(prc),
                                     out["res"].data_ptr(), out["bound_idx"].data_ptr(), out["phi"].data_ptr(),
                                     out["removed_iter"].data_ptr(),
                                     None if error_out is None else error_out.data_ptr(), stream)
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
                                     None, None, None, None, None, None)
    assert rc == ahf.ERR_INVALID
    assert b"AHF_STATIC_MAX_HALOS" in lib.ahf_last_error()
    one = ahf.halos_from_population(pop)
    one["count"][0] = ahf.STATIC_MAX_COUNT + 1
    dummy = np.zeros(16, dtype=np.int64)
    rc = lib.ahf_unbind_batch_static(ctypes.byref(pc), one.ctypes.data, len(one), None, ctypes.byref(prc),
                                     dummy.ctypes.data, dummy.ctypes.data, None, None, None, None)
    assert rc == ahf.ERR_INVALID
    assert b"AHF_STATIC_MAX_COUNT" in lib.ahf_last_error()


def _agree(pop, ref, out):
    """The static call's outputs against ahf_unbind_batch's on the same inputs."""
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
    # batches of different shapes, every halo within the on-chip class: float32
    # relative coordinates; float64 with masses; a member list with the
    # density-rise edge variant; float32 box coordinates in a periodic box
    tail = synth.large_tail(seed=24, n_halos=3, n_lo=1500, n_hi=7000, n_sub=3, box=5e5)
    member_pop = synth.halo_batch(seed=25, n_halos=12, n_lo=200, n_hi=6000)
    rng = np.random.default_rng(26)
    members = np.concatenate([rng.permutation(np.arange(o, o + c)) for o, c in
                              zip(member_pop.offset, member_pop.count)]).astype(np.int64)
    cases = [(synth.halo_batch(seed=22, n_halos=40, n_lo=100, n_hi=7000), {}, None),
             (synth.halo_batch(seed=23, n_halos=17, n_lo=300, n_hi=7000, coord_type=synth.COORD_F64,
                               with_masses=True), {}, None),
             (member_pop, {"variant": ahf.VAR_RISE_EDGE}, members),
             (tail, {}, None)]
    for pop, _, _ in cases:
        assert pop.count.max() <= ahf.STATIC_MAX_COUNT
    runs = []
    for pop, kw, mi in cases:
        parts = ahf.particles_from_population(pop)
        hal = ahf.halos_from_population(pop)
        prm = ahf.params_for(pop, **kw)
        mi_dev = None if mi is None else torch.from_numpy(mi).cuda()
        ref = ctx.unbind_batch(parts, hal, prm, member_idx=mi_dev, stream=stream)
        out = ctx.alloc_outputs(len(hal), pop.n_particles)
        err = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        runs.append((pop, parts, hal, prm, mi_dev, ref, out, err))
    torch.cuda.synchronize()
    # two rounds of every batch back to back on one stream: the first round
    # also sets up the device (the scratch address, and the kernels' code,
    # which the driver may load at a kernel's first launch); the second takes
    # no device memory at all
    free0 = None
    for _ in range(2):
        for pop, parts, hal, prm, mi_dev, ref, out, err in runs:
            rc = _call_static(parts, hal, prm, out, stream.cuda_stream, mi_dev, err)
            assert rc == ahf.OK, ahf.load_library().ahf_last_error()
        torch.cuda.synchronize()
        if free0 is None:
            free0 = torch.cuda.mem_get_info()[0]
    assert torch.cuda.mem_get_info()[0] == free0
    for pop, parts, hal, prm, mi_dev, ref, out, err in runs:
        assert int(err.item()) == ahf.OK
        _agree(pop, ref, out)


@pytest.mark.gpu
def test_static_reports_bad_member_index_and_refuses_capture():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_3662_gb300 import build_lib
    build_lib.build()
    torch.cuda.set_device(0)
    ctx = ahf.Context(0)
    pop = synth.halo_batch(seed=27, n_halos=6, n_lo=200, n_hi=3000)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    mi = np.arange(pop.n_particles, dtype=np.int64)
    mi[int(pop.offset[2]) + 5] = pop.n_particles + 10          # out of range: a non-member, reported
    mi_dev = torch.from_numpy(mi).cuda()
    out = ctx.alloc_outputs(len(hal), pop.n_particles)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    assert _call_static(parts, hal, prm, out, stream.cuda_stream, mi_dev, err) == ahf.OK
    torch.cuda.synchronize()
    assert int(err.item()) == ahf.ERR_INVALID
    assert int(out["removed_iter"].cpu().numpy()[int(pop.offset[2]) + 5]) == -1
    # the next call starts with a clean error word
    assert _call_static(parts, hal, prm, out, stream.cuda_stream, None, err) == ahf.OK
    torch.cuda.synchronize()
    assert int(err.item()) == ahf.OK
    # while its stream is being captured the call refuses and enqueues nothing
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = _call_static(parts, hal, prm, out, side.cuda_stream, None, err)
    assert rc == ahf.ERR_INVALID
    assert b"captured" in ahf.load_library().ahf_last_error()

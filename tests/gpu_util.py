"""Helpers for the GPU tests: build once, run the C ABI, fetch outputs."""
import numpy as np
import pytest

_built = False


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    global _built
    if not _built:
        from paper_0904_3662_gb300 import build_lib
        build_lib.build()
        _built = True
    return torch


def run_gpu(pop, params=None, halos=None, member_idx=None, plain=False, ctx=None, **kw):
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    if ctx is None:
        ctx = ahf.Context(0)
        # the smallest class per halo, so that each test exercises the classes
        # its sizes select (promotion of small batches has its own tests)
        ctx.set_option(ahf.OPT_PROMOTE, 0)
    parts = ahf.particles_from_population(pop)
    prm = params or ahf.params_for(pop)
    hal = ahf.halos_from_population(pop) if halos is None else halos
    mi = None if member_idx is None else torch.from_numpy(member_idx).cuda()
    out = ctx.unbind_batch(parts, hal, prm, member_idx=mi, plain=plain, **kw)
    torch.cuda.synchronize()
    ctx.sync()
    host = {
        "res": ahf.results_to_numpy(out["res"]),
        "bound_idx": out["bound_idx"].cpu().numpy(),
        "phi": None if out["phi"] is None else out["phi"].cpu().numpy(),
        "removed_iter": None if out["removed_iter"] is None else out["removed_iter"].cpu().numpy(),
    }
    return host, prm, ctx, out

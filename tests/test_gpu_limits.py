"""Limits a caller sets on a context: the bounded wait of the multi-CTA
passes (AHF_OPT_WAIT_LIMIT: a warp that gives up waiting for its tensor copy
reports AHF_ERR_TIMEOUT through ahf_sync, and the context stays usable) and
the workspace cap (AHF_OPT_WORKSPACE_CAP: a call that needs more fails with
AHF_ERR_NOMEM before enqueuing anything).  The failure is made on purpose by
a limit of zero polls, never by a fault."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu
from tests.parity import compare

pytestmark = pytest.mark.gpu


def _pop():
    # one host above the on-chip classes (the multi-CTA passes with tensor
    # copies: mixed mode, uniform mass) and a few small haloes
    return synth.large_tail(seed=63, counts=[300_000, 2_000, 9_000], n_sub=4, box=5e5)


def test_wait_limit_zero_reports_timeout_and_the_context_recovers():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = _pop()
    ctx = ahf.Context(0)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    ctx.set_option(ahf.OPT_WAIT_LIMIT, 0)
    assert ctx.get_option(ahf.OPT_WAIT_LIMIT) == 0
    ctx.unbind_batch(parts, hal, prm)
    torch.cuda.synchronize()
    with pytest.raises(ahf.AHFError) as e:
        ctx.sync()
    assert e.value.code == ahf.ERR_TIMEOUT
    ctx.sync()                                   # the error word was cleared
    # the same context with the default limit: correct results
    ctx.set_option(ahf.OPT_WAIT_LIMIT, 1 << 22)
    out = ctx.unbind_batch(parts, hal, prm)
    torch.cuda.synchronize()
    ctx.sync()
    compare(pop, prm, ahf.results_to_numpy(out["res"]), out["bound_idx"].cpu().numpy(), out["phi"].cpu().numpy(),
            out["removed_iter"].cpu().numpy())


def test_workspace_cap_refuses_a_larger_call():
    torch = require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = _pop()
    ctx = ahf.Context(0)
    ctx.set_option(ahf.OPT_WORKSPACE_CAP, 1 << 20)
    parts = ahf.particles_from_population(pop)
    hal = ahf.halos_from_population(pop)
    prm = ahf.params_for(pop)
    with pytest.raises(ahf.AHFError) as e:
        ctx.unbind_batch(parts, hal, prm)
    assert e.value.code == ahf.ERR_NOMEM
    assert b"cap" in ahf.load_library().ahf_last_error()
    ctx.set_option(ahf.OPT_WORKSPACE_CAP, 0)
    out = ctx.unbind_batch(parts, hal, prm)
    torch.cuda.synchronize()
    ctx.sync()
    res = ahf.results_to_numpy(out["res"])
    assert np.all(res["n_bound"] > 0)

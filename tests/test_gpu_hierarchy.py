"""Hosts and subhaloes unbound in dependency order (Sect. 2.1) on the GPU
against the oracle's hierarchical unbinding."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu
from tests.parity import compare
from tests.test_oracle_variants import _host_with_subhaloes

pytestmark = pytest.mark.gpu


def _run(ctx, pop, parent, member_idx, prm):
    import torch
    from paper_0904_3662_gb300 import ahf
    parts = ahf.particles_from_population(pop)
    mi = None if member_idx is None else torch.from_numpy(member_idx).cuda()
    out = ctx.unbind_hierarchy(parts, ahf.halos_from_population(pop), parent, prm, member_idx=mi)
    torch.cuda.synchronize()
    ctx.sync()
    return {"res": ahf.results_to_numpy(out["res"]), "bound_idx": out["bound_idx"].cpu().numpy(),
            "phi": out["phi"].cpu().numpy(), "removed_iter": out["removed_iter"].cpu().numpy()}


@pytest.mark.parametrize("precision", [0, 1])
def test_host_with_subhaloes(precision):
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop, member_idx, parent = _host_with_subhaloes()
    prm = ahf.params_for(pop, precision=precision)
    ctx = ahf.Context(0)
    g = _run(ctx, pop, parent, member_idx, prm)
    compare(pop, prm, g["res"], g["bound_idx"], g["phi"], g["removed_iter"], member_idx=member_idx,
            parent=parent, phi_rtol=1e-11 if precision else 1e-5, exact_order=bool(precision))
    # the subhaloes' particles leave the host: fewer members than the flat run
    import torch
    flat = ctx.unbind_batch(ahf.particles_from_population(pop), ahf.halos_from_population(pop), prm,
                            member_idx=torch.from_numpy(member_idx).cuda())
    torch.cuda.synchronize()
    fr = ahf.results_to_numpy(flat["res"])
    assert g["res"]["n_member"][0] < fr["n_member"][0]
    assert g["res"]["n_member"][4] == fr["n_member"][4]          # the deepest level is unchanged


def test_forest_of_batch_haloes_and_errors():
    """Disjoint haloes with an arbitrary forest over them: the exclusions
    only touch particles a descendant bound, which here are nobody's else."""
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.halo_batch(seed=97, n_halos=30, n_lo=100, n_hi=40_000)
    rng = np.random.default_rng(3)
    parent = np.array([-1 if h < 5 else int(rng.integers(0, h)) for h in range(pop.n_halos)])
    prm = ahf.params_for(pop)
    ctx = ahf.Context(0)
    g = _run(ctx, pop, parent, None, prm)
    compare(pop, prm, g["res"], g["bound_idx"], g["phi"], g["removed_iter"], parent=parent)
    # a forest that is flat is the batch call
    flat = _run(ctx, pop, np.full(pop.n_halos, -1), None, prm)
    compare(pop, prm, flat["res"], flat["bound_idx"], flat["phi"], flat["removed_iter"])
    for bad in (np.r_[1, 0, np.full(pop.n_halos - 2, -1)], np.r_[pop.n_halos, np.full(pop.n_halos - 1, -1)]):
        with pytest.raises(ahf.AHFError) as e:
            _run(ctx, pop, bad, None, prm)
        assert e.value.code == ahf.ERR_INVALID

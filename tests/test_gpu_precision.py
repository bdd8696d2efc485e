"""Precision sweep at its full size: 1e5 haloes of the batch law (N_p ~ N^-1.9
on [1e2, 1e5], 10 % background, float64 inputs, ~1.0e8 particles), every halo
unbound in the mixed mode (FP32 per-particle arithmetic, exact fixed-point
sums) and in the all-FP64 mode, and every halo compared with the FP64 oracle
(spread over the host cores).  Prints the worst relative errors of phi, M_vir
and R_vir, the worst radial-order inversion and the band-set size (run with
-s to see the table)."""
import time

import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu
from tests.oracle_pool import compare_parallel
from tests.parity import fp64_rtol

pytestmark = pytest.mark.gpu


def test_precision_sweep_full_size_both_modes():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    t0 = time.perf_counter()
    pop = synth.precision_sweep()
    assert pop.n_halos == 100_000
    rows = []
    for name, prec, tol, exact in (("mixed", ahf.PREC_MIXED, 1e-5, False), ("fp64", ahf.PREC_FP64, fp64_rtol(pop), True)):
        prm = ahf.params_for(pop, precision=prec)
        out, prm, ctx, _ = run_gpu(pop, params=prm)
        res = out["res"]
        s = compare_parallel(pop, prm, res, out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=tol,
                             vir_rtol=tol, exact_order=exact)
        assert s["halos"] == pop.n_halos
        rows.append((name, s["halos"], int(res["n_member"].sum()), int(res["part_iter"].sum()), s["worst_phi_rel"],
                     s["worst_vir_rel"], s["worst_order_inversion"], s["n_band"]))
        assert s["worst_phi_rel"] <= tol and s["worst_vir_rel"] <= tol
        assert np.all(res["status"] & ahf.HALO_NOT_CONVERGED == 0)
    print(f"\nprecision sweep: {pop.n_particles} particles, {time.perf_counter() - t0:.0f} s")
    print("mode   haloes  members    particle-iterations  worst |dphi/phi|  worst |dM/M|,|dR/R|  "
          "worst order inversion  band tests")
    for r in rows:
        print(f"{r[0]:6s} {r[1]:6d} {r[2]:10d} {r[3]:20d}  {r[4]:16.3e}  {r[5]:19.3e}  {r[6]:21.3e}  {r[7]:10d}")

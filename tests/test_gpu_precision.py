"""Precision sweep: the 1e5-halo population's law (N_p ~ N^-1.9 on [1e2, 1e5],
10 % background, float64 inputs) at 5,000 haloes, every halo unbound in the
mixed mode (FP32 per-particle arithmetic, exact fixed-point sums) and in the
all-FP64 mode, each compared halo by halo with the FP64 oracle.  Prints the
worst relative errors of phi, M_vir and R_vir and the band-set size (run
with -s to see the table)."""
import numpy as np
import pytest

from paper_0904_3662_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu
from tests.parity import compare

pytestmark = pytest.mark.gpu

N_HALOS = 5000


def test_precision_sweep_mixed_and_fp64():
    require_gpu()
    from paper_0904_3662_gb300 import ahf
    pop = synth.precision_sweep(n_halos=N_HALOS)
    rows = []
    for name, prec, tol, exact in (("mixed", ahf.PREC_MIXED, 1e-5, False), ("fp64", ahf.PREC_FP64, 1e-11, True)):
        prm = ahf.params_for(pop, precision=prec)
        out, prm, ctx, _ = run_gpu(pop, params=prm)
        s = compare(pop, prm, out["res"], out["bound_idx"], out["phi"], out["removed_iter"], phi_rtol=tol,
                    vir_rtol=tol, exact_order=exact)
        res = out["res"]
        rows.append((name, s["halos"], int(res["n_member"].sum()), int(res["part_iter"].sum()), s["worst_phi_rel"],
                     s["worst_vir_rel"], s["n_band"]))
        assert s["worst_phi_rel"] <= tol and s["worst_vir_rel"] <= tol
    print("\nmode   haloes  members   particle-iterations  worst |dphi/phi|  worst |dM_vir/M_vir|,|dR/R|  band tests")
    for r in rows:
        print(f"{r[0]:6s} {r[1]:6d} {r[2]:9d} {r[3]:20d}  {r[4]:16.3e}  {r[5]:27.3e}  {r[6]:10d}")

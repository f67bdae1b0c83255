"""Every precision form at the precision configuration, against FP64 of the ORIGINAL values.

16,384 x 16,384 at 90% (uniform rows, and clustered 16 x 8 blocks at 40% fill), SpMM N = 256
and SDDMM Kd = 256, dense operands N(0, 1) and A's values U[-1, 1).  Each form quantises the
FP32 inputs with the library's roundings (bit-exact against the oracle's elsewhere), runs
its kernels, and is compared on 400 sampled rows with the FP64 oracle run on the original
FP32 values, so the error includes the quantisation.  Tolerances per output, scaled by
sum |a||b|: FP32 1e-5, BF16 1e-2, FP8-E4M3 4e-2 (tensor-core forms included).
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 1e-2, "e4m3": 4e-2, "tc_bf16": 1e-2, "tc_e4m3": 4e-2}
N = 256


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


@pytest.fixture(scope="module", params=["uniform", "clustered"])
def case(request, gb):
    import torch

    A = (gen.csr_uniform(16384, 16384, 0.9, seed=2001) if request.param == "uniform"
         else gen.csr_clustered(16384, 16384, 0.9, seed=2002))
    B, X, Y = (gen.dense_normal(16384, N, 2003 + k) for k in range(3))
    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    Bd, Xd, Yd = dev(B), dev(X), dev(Y)
    wins = np.sort(np.random.default_rng(17).choice(A.M // 16, 25, replace=False))
    rows = (wins[:, None] * 16 + np.arange(16)).ravel()
    srp, sci, sv, idx = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    ref_c, sc_c = oracle.spmm(srp, sci, sv, B)
    ref_o, sc_o = oracle.sddmm(srp, sci, sv, X[rows], Y)
    yield dict(name=request.param, A=A, rp=rp, ci=ci, v=v, Bd=Bd, Xd=Xd, Yd=Yd, rows=rows, idx=idx,
               ref_c=ref_c, sc_c=sc_c, ref_o=ref_o, sc_o=sc_o)
    del rp, ci, v, Bd, Xd, Yd
    torch.cuda.empty_cache()


def _run(gb, c, form):
    rp, ci, v, Bd, Xd, Yd, K = c["rp"], c["ci"], c["v"], c["Bd"], c["Xd"], c["Yd"], c["A"].K
    if form == "fp32":
        return gb.spmm(rp, ci, v, Bd), gb.sddmm(rp, ci, v, Xd, Yd)
    if form in ("bf16", "tc_bf16"):
        qa, qb, qx, qy = (gb.quantize_bf16(t) for t in (v, Bd, Xd, Yd))
        if form == "bf16":
            return gb.spmm(rp, ci, qa, qb), gb.sddmm(rp, ci, v, qx, qy)
        plan = gb.TcPlan(rp, ci, qa, K)
        C, out = plan.execute(qb), plan.sddmm(v, qx, qy)
        plan.check()
        plan.close()
        return C, out
    ea, sa = gb.quantize_e4m3_rows(v, rp)
    (eb, sb), (ex, ux), (ey, uy) = (gb.quantize_e4m3_rows(t) for t in (Bd, Xd, Yd))
    if form == "e4m3":
        return (gb.spmm(rp, ci, ea, eb, a_scale=sa, b_scale=sb),
                gb.sddmm(rp, ci, v, ex, ey, x_scale=ux, y_scale=uy))
    plan = gb.TcPlan(rp, ci, ea, K, row_scale=sa)
    C, out = plan.execute(eb, row_scale=sb), plan.sddmm(v, ex, ey, x_scale=ux, y_scale=uy)
    plan.check()
    plan.close()
    return C, out


@pytest.mark.parametrize("form", list(TOL))
def test_precision_form_against_fp64_of_original_values(gb, case, form):
    C, out = _run(gb, case, form)
    C, out = C.cpu().numpy(), out.cpu().numpy()
    tol = TOL[form]
    e_c = assert_within(C[case["rows"]], case["ref_c"], case["sc_c"], tol, f"{case['name']} {form} spmm")
    e_o = assert_within(out[case["idx"]], case["ref_o"], case["sc_o"], tol, f"{case['name']} {form} sddmm")
    print(f"\n{case['name']} {form}: spmm err max {e_c[0]:.3e} mean {e_c[1]:.3e}; "
          f"sddmm err max {e_o[0]:.3e} mean {e_o[1]:.3e} (tolerance {tol:g})")

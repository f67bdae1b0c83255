"""GPU parity of the K-range-binned SpMM plan (Eq. 1 summed slice by slice).

C = A B with A's columns cut into slices of W consecutive indices; pass 0 writes each row's
part from the first slice, later passes add theirs.  Integer inputs (every partial sum
exact in FP32) must match the FP64 oracle bit for bit for any slice width; random FP32
inputs are held to the FP32 tolerance, 1e-5 of sum |a||b| per output.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def plan_of(gb, A, vals=None, N=64, slice_cols=0):
    return gb.KbinPlan(dev(A.rowptr), dev(A.colidx), dev(A.vals if vals is None else vals), A.K, N, slice_cols)


@pytest.mark.parametrize("slice_cols", [0, 2, 7, 64, 1000, 4099])
@pytest.mark.parametrize("N", [4, 32, 64, 128, 200])
def test_kbin_integers_bit_exact(gb, slice_cols, N):
    """K = 4099 (no slice width divides it), rows of about 41 entries."""
    A = gen.csr_uniform(2000, 4099, 0.99, seed=601)
    vals = gen.vals_int(A.nnz, 602)
    B = gen.dense_int(A.K, N, 603)
    plan = plan_of(gb, A, vals, N, slice_cols)
    W = plan.info()["slice_cols"]
    assert plan.info()["slices"] == -(-A.K // W)
    C = plan.execute(dev(B)).cpu().numpy()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("layout", ["uniform", "powerlaw"])
@pytest.mark.parametrize("slice_cols", [0, 5000])
def test_kbin_random_fp32(gb, layout, slice_cols):
    make = gen.csr_uniform if layout == "uniform" else gen.csr_powerlaw
    A = make(3000, 50000, 0.995, seed=604)
    B = gen.dense_normal(A.K, 64, 605)
    plan = plan_of(gb, A, N=64, slice_cols=slice_cols)
    C = plan.execute(dev(B)).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL32, f"kbin {layout}")


def test_kbin_auto_slice_width(gb):
    """slice_cols = 0: the B rows of width N that fill 48 MB (at least 1024), capped at K."""
    A = gen.csr_uniform(64, 300000, 0.999, seed=606)
    for N, W in ((128, (48 << 20) // 512), (64, (48 << 20) // 256), (4096, 3072)):
        info = plan_of(gb, A, N=N).info()
        assert info["slice_cols"] == min(max(W, 1024), A.K)
        assert info["slices"] == -(-A.K // info["slice_cols"])
    small = gen.csr_uniform(64, 500, 0.9, seed=607)
    assert plan_of(gb, small).info() == {"slices": 1, "slice_cols": 500, "rows": 64, "nnz": small.nnz}


def test_kbin_edge_cases(gb):
    import torch

    rng = np.random.default_rng(608)
    # empty rows, repeated (non-decreasing) column indices, rows living in the last slice only
    lengths = rng.integers(0, 30, 500)
    lengths[:100] = 0
    A = gen.csr_from_lengths(lengths, 3000, seed=609)
    rows = np.concatenate([np.repeat(np.arange(A.M), A.row_lengths()), [200, 200, 200, 300, 300]])
    cols = np.concatenate([A.colidx, [11, 11, 11, 2999, 2999]])
    order = np.lexsort((cols, rows))  # by row, then column: repeats adjacent, rows sorted
    R = gen.csr_from_triplets(A.M, A.K, rows[order], cols[order], gen.vals_int(A.nnz + 5, 610))
    assert R.row_lengths()[200] >= 3 and np.count_nonzero(R.colidx == 2999) >= 2
    B = gen.dense_int(R.K, 32, 611)
    for sc in (0, 1, 100, 2999):
        C = plan_of(gb, R, N=32, slice_cols=sc).execute(dev(B)).cpu().numpy()
        want, _ = oracle.spmm(R.rowptr, R.colidx, R.vals, B)
        assert np.array_equal(C.astype(np.float64), want)
    # no stored entries at all: C is zero
    Z = gen.csr_from_lengths(np.zeros(50, np.int64), 100, seed=612)
    C = plan_of(gb, Z, N=8, slice_cols=10).execute(dev(gen.dense_int(100, 8, 613))).cpu().numpy()
    assert np.all(C == 0)
    # no rows; N = 0
    empty = gb.KbinPlan(torch.zeros(1, dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.float32, device="cuda"), 10, 8)
    assert empty.execute(dev(gen.dense_int(10, 8, 614))).shape == (0, 8)
    out = plan_of(gb, A, N=0).execute(torch.zeros((A.K, 0), device="cuda"))
    assert out.shape == (A.M, 0)


def test_kbin_values_in_place_and_padded_ld(gb):
    """The plan keeps A's pointers: new values in the same buffer are used; B and C with
    leading dimensions above N."""
    import torch

    A = gen.csr_uniform(1000, 8000, 0.99, seed=615)
    v = dev(gen.vals_int(A.nnz, 616))
    plan = gb.KbinPlan(dev(A.rowptr), dev(A.colidx), v, A.K, 64, 1500)
    Bw = dev(gen.dense_int(A.K, 72, 617))
    Cw = torch.full((A.M, 72), 7.0, device="cuda")
    for seed in (618, 619):
        vals = gen.vals_int(A.nnz, seed)
        v.copy_(dev(vals))
        plan.execute(Bw[:, :64], out=Cw[:, :64])
        want, _ = oracle.spmm(A.rowptr, A.colidx, vals, Bw[:, :64].cpu().numpy())
        assert np.array_equal(Cw[:, :64].cpu().numpy().astype(np.float64), want)
    assert torch.all(Cw[:, 64:] == 7.0)


def test_kbin_argument_errors(gb):
    import torch

    A = gen.csr_uniform(100, 5000, 0.99, seed=620)
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):  # 5000 slices of one column
        plan_of(gb, A, slice_cols=1)
    bad = A.colidx.copy()
    r = int(np.argmax(A.row_lengths() >= 2))
    p = A.rowptr[r]
    bad[p], bad[p + 1] = bad[p + 1], bad[p]  # one row out of order
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        gb.KbinPlan(dev(A.rowptr), dev(bad), dev(A.vals), A.K, 64)
    out_of_range = A.colidx.copy()
    out_of_range[-1] = A.K
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        gb.KbinPlan(dev(A.rowptr), dev(out_of_range), dev(A.vals), A.K, 64)
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):  # BF16 values
        gb.KbinPlan(dev(A.rowptr), dev(A.colidx), dev(A.vals).to(torch.bfloat16), A.K, 64)
    plan = plan_of(gb, A)
    with pytest.raises(gb.GbspError, match="ALIGN"):  # N not a multiple of 4
        plan.execute(torch.zeros((A.K, 6), device="cuda"))
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):  # B rows != K
        plan.execute(torch.zeros((A.K + 1, 8), device="cuda"))


def test_kbin_full_size_sampled_rows(gb):
    """1,048,576^2 at 99.99% (about 110M nonzeros), N = 128, default slices (the launch the
    bench times): 400 sampled rows against the oracle."""
    A = gen.csr_uniform(1048576, 1048576, 0.9999, seed=1003)
    B = gen.dense_normal(A.K, 128, 621)
    plan = plan_of(gb, A, N=128)
    assert plan.info()["slices"] == 11
    C = plan.execute(dev(B))
    rows = np.sort(np.random.default_rng(14).choice(A.M, 400, replace=False))
    got = C[dev(rows.astype(np.int64))].cpu().numpy()
    rp, ci, v, _ = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    ref, sc = oracle.spmm(rp, ci, v, B)
    assert_within(got, ref, sc, TOL32, "kbin full size")

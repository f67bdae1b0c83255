"""GPU parity of the hyper-sparse SpMM plan (Eq. 1 with rows binned by length).

Rows with more than 32 entries run as in the row split, rows with 1 to 32 entries one per
lane group, empty rows give zero C rows.  Integer inputs must match the FP64 oracle bit
for bit; random FP32 inputs are held to 1e-5 of sum |a||b| per output.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def mixed_lengths(M, seed):
    """60% empty rows, 30% with 1-4 entries, 8% with 5-32, 2% with 33-300."""
    rng = np.random.default_rng(seed)
    kind = rng.random(M)
    lengths = np.zeros(M, np.int64)
    lengths[(kind >= 0.6) & (kind < 0.9)] = rng.integers(1, 5, M)[(kind >= 0.6) & (kind < 0.9)]
    lengths[(kind >= 0.9) & (kind < 0.98)] = rng.integers(5, 33, M)[(kind >= 0.9) & (kind < 0.98)]
    lengths[kind >= 0.98] = rng.integers(33, 301, M)[kind >= 0.98]
    return lengths


def plan_of(gb, A, vals=None):
    return gb.HspPlan(dev(A.rowptr), dev(A.colidx), dev(A.vals if vals is None else vals), A.K)


@pytest.mark.parametrize("N", [4, 8, 32, 64, 128, 200, 516])
def test_hsp_integers_bit_exact(gb, N):
    A = gen.csr_from_lengths(mixed_lengths(5000, 701), 3000, seed=702)
    vals = gen.vals_int(A.nnz, 703)
    B = gen.dense_int(A.K, N, 704)
    plan = plan_of(gb, A, vals)
    lens = A.row_lengths()
    assert plan.info() == {"long_rows": int(np.sum(lens > 32)), "short_rows": int(np.sum((lens > 0) & (lens <= 32))),
                           "empty_rows": int(np.sum(lens == 0)), "nnz": A.nnz}
    C = plan.execute(dev(B)).cpu().numpy()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("case", ["uniform_2_per_row", "uniform_1_per_row", "powerlaw"])
def test_hsp_random_fp32(gb, case):
    if case == "uniform_2_per_row":
        A = gen.csr_uniform(20000, 20000, 0.9999, seed=705)
    elif case == "uniform_1_per_row":
        A = gen.csr_uniform(50000, 50000, 0.99998, seed=706)
    else:
        A = gen.csr_powerlaw(20000, 20000, 0.9995, seed=707)
    B = gen.dense_normal(A.K, 64, 708)
    C = plan_of(gb, A).execute(dev(B)).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL32, f"hsp {case}")


def test_hsp_edge_cases(gb):
    import torch

    # unsorted and repeated column indices in short and long rows
    rng = np.random.default_rng(709)
    lengths = mixed_lengths(800, 710)
    rows = np.repeat(np.arange(800), lengths)
    cols = rng.integers(0, 50, rows.size)  # repeats likely, order random
    R = gen.csr_from_triplets(800, 50, rows, cols, gen.vals_int(rows.size, 711), sort=True)
    B = gen.dense_int(50, 32, 712)
    C = plan_of(gb, R).execute(dev(B)).cpu().numpy()
    want, _ = oracle.spmm(R.rowptr, R.colidx, R.vals, B)
    assert np.array_equal(C.astype(np.float64), want)
    # no stored entries: C is zero, whatever it held
    Z = gen.csr_from_lengths(np.zeros(300, np.int64), 40, seed=713)
    out = torch.full((300, 16), 3.0, device="cuda")
    plan_of(gb, Z).execute(dev(gen.dense_int(40, 16, 714)), out=out)
    assert torch.all(out == 0)
    # one long row only; no rows; N = 0
    L = gen.csr_from_lengths(np.array([0, 700, 0]), 1000, seed=715)
    Lv = gen.vals_int(L.nnz, 726)
    Bl = gen.dense_int(1000, 64, 716)
    want, _ = oracle.spmm(L.rowptr, L.colidx, Lv, Bl)
    assert np.array_equal(plan_of(gb, L, Lv).execute(dev(Bl)).cpu().numpy().astype(np.float64), want)
    empty = gb.HspPlan(torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                       torch.zeros(0, dtype=torch.float32, device="cuda"), 10)
    assert empty.execute(dev(gen.dense_int(10, 8, 717))).shape == (0, 8)
    assert plan_of(gb, L).execute(torch.zeros((1000, 0), device="cuda")).shape == (3, 0)


def test_hsp_values_in_place_and_padded_ld(gb):
    import torch

    A = gen.csr_from_lengths(mixed_lengths(2000, 718), 4000, seed=719)
    v = dev(gen.vals_int(A.nnz, 720))
    plan = gb.HspPlan(dev(A.rowptr), dev(A.colidx), v, A.K)
    Bw = dev(gen.dense_int(A.K, 136, 721))
    Cw = torch.full((A.M, 136), 5.0, device="cuda")
    for seed in (722, 723):
        vals = gen.vals_int(A.nnz, seed)
        v.copy_(dev(vals))
        plan.execute(Bw[:, :128], out=Cw[:, :128])
        want, _ = oracle.spmm(A.rowptr, A.colidx, vals, Bw[:, :128].cpu().numpy())
        assert np.array_equal(Cw[:, :128].cpu().numpy().astype(np.float64), want)
    assert torch.all(Cw[:, 128:] == 5.0)


def test_hsp_argument_errors(gb):
    import torch

    A = gen.csr_from_lengths(mixed_lengths(300, 724), 500, seed=725)
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):  # BF16 values
        gb.HspPlan(dev(A.rowptr), dev(A.colidx), dev(A.vals).to(torch.bfloat16), A.K)
    bad = A.colidx.copy()
    bad[0] = A.K
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        gb.HspPlan(dev(A.rowptr), dev(bad), dev(A.vals), A.K)
    plan = plan_of(gb, A)
    with pytest.raises(gb.GbspError, match="ALIGN"):
        plan.execute(torch.zeros((A.K, 6), device="cuda"))
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):
        plan.execute(torch.zeros((A.K - 1, 8), device="cuda"))


def test_hsp_plan_created_on_nonblocking_stream(gb):
    """Plan creation uploads its row lists and records on the caller's stream; on a
    non-blocking side stream (which does not order against the legacy default stream) the
    first execution on that stream must still see every record."""
    import torch

    A = gen.csr_from_lengths(mixed_lengths(20000, 481), 3000, seed=482)
    vals = gen.vals_int(A.nnz, 483)
    B = gen.dense_int(A.K, 64, 484)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(vals), dev(B)
        plan = gb.HspPlan(rp, ci, v, A.K, stream=side)
        C = plan.execute(Bd, stream=side)
    side.synchronize()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), want)
    plan.close()

"""GPU parity of the FP32 SpMM (Eq. 1) and SDDMM (Eq. 2) kernels against the FP64 oracle.

Tolerance (FP32 path): |gpu - oracle| <= 1e-5 * sum |a||b| per output (sum |s||x||y| for
SDDMM); outputs whose scale is 0 must be exactly 0.  Integer-valued inputs must match the
oracle bit for bit (every partial sum is an exact integer below 2^24).
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def _dup_unsorted(seed=0):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(40):
        L = int(rng.integers(0, 12))
        c = list(rng.integers(0, 30, L))  # repeats allowed, unsorted
        rows += [i] * L
        cols += c
    return gen.csr_from_triplets(40, 30, rows, cols, rng.uniform(-1, 1, len(cols)), sort=True)


def _one_dense_row():
    lengths = np.full(300, 3)
    lengths[17] = 2000
    lengths[250] = 0
    return gen.csr_from_lengths(lengths, 2000, seed=9)


MATS = {
    "uniform1024": lambda: gen.csr_uniform(1024, 1024, 0.9, seed=0),
    "powerlaw": lambda: gen.csr_powerlaw(3000, 2500, 0.99, seed=3),
    "hypersparse": lambda: gen.csr_uniform(6000, 6000, 0.9999, seed=4),
    "ragged": lambda: gen.csr_uniform(37, 53, 0.7, seed=5),
    "dup_unsorted": _dup_unsorted,
    "dense_row": _one_dense_row,
}
_cache = {}


def mat(name):
    if name not in _cache:
        _cache[name] = MATS[name]()
    return _cache[name]


def run_spmm(gb, A, B, **kw):
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), **kw)
    return C.cpu().numpy()


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("N", [4, 16, 32, 64, 68, 96, 128, 132, 256, 264])
@pytest.mark.parametrize("variant", ["rowsplit", "merge"])
def test_spmm_fp32(gb, name, N, variant):
    A = mat(name)
    B = gen.dense_normal(A.K, N, 11)
    C = run_spmm(gb, A, B, variant=variant)
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, scale, TOL, f"{name} N={N} {variant}")


@pytest.mark.parametrize("vecs", [1, 2, 4])
@pytest.mark.parametrize("unroll", [1, 2, 4, 8])
@pytest.mark.parametrize("variant", ["rowsplit", "merge"])
def test_spmm_layouts(gb, vecs, unroll, variant):
    """Every (vectors per lane, gathers in flight) layout on full and partial column tiles."""
    A = mat("powerlaw")
    for N in (8, 64, 96, 128, 264):
        B = gen.dense_normal(A.K, N, 12)
        C = run_spmm(gb, A, B, variant=variant, unroll=unroll, vecs=vecs)
        ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
        assert_within(C, ref, scale, TOL, f"vecs={vecs} unroll={unroll} N={N}")


@pytest.mark.parametrize("ctas", [1, 2, 7])
def test_spmm_merge_grid_shapes(gb, ctas):
    """Small merge-path grids split long rows across many warps (carry fix-up path)."""
    A = mat("dense_row")
    B = gen.dense_normal(A.K, 64, 13)
    C = run_spmm(gb, A, B, variant="merge", ctas_per_sm=ctas)
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, scale, TOL, f"ctas={ctas}")


@pytest.mark.parametrize("N", [1, 3, 33, 130])
def test_spmm_scalar_any_width(gb, N):
    A = mat("powerlaw")
    B = gen.dense_normal(A.K, N, 14)
    C = run_spmm(gb, A, B)  # auto picks the unvectorised kernel
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, scale, TOL, f"scalar N={N}")
    with pytest.raises(gb.GbspError, match="ALIGN"):
        run_spmm(gb, A, B, variant="rowsplit")


def test_spmm_padded_leading_dimension(gb):
    import torch

    A = mat("uniform1024")
    Bfull = gen.dense_normal(A.K, 80, 15)
    Bv = dev(Bfull)[:, :64]  # ld = 80
    Cfull = torch.full((A.M, 72), 7.0, device="cuda")
    Cv = Cfull[:, :64]
    gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), Bv, out=Cv)
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, Bfull[:, :64])
    assert_within(Cv.cpu().numpy(), ref, scale, TOL, "ld")
    assert torch.all(Cfull[:, 64:] == 7.0), "columns past N untouched"


@pytest.mark.parametrize("variant", ["rowsplit", "merge", "scalar"])
def test_spmm_integers_bit_exact(gb, variant):
    A = gen.csr_powerlaw(2000, 1500, 0.98, seed=21)
    A = A.with_vals(gen.vals_int(A.nnz, 22))
    B = gen.dense_int(A.K, 64, 23)
    C = run_spmm(gb, A, B, variant=variant)
    ref, _ = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert np.array_equal(C.astype(np.float64), ref)


def test_spmm_identity_bit_exact(gb):
    K = 777
    A = gen.csr_from_triplets(K, K, np.arange(K), np.arange(K), np.ones(K))
    B = gen.dense_normal(K, 64, 24)
    for variant in ("rowsplit", "merge"):
        assert np.array_equal(run_spmm(gb, A, B, variant=variant), B)


def test_spmm_empty_and_degenerate(gb):
    import torch

    # no stored entries at all: C is all zeros (and overwritten, not accumulated)
    A = gen.csr_from_lengths(np.zeros(50, dtype=np.int64), 20, seed=1)
    B = gen.dense_normal(20, 32, 2)
    out = torch.full((50, 32), 3.0, device="cuda")
    for variant in ("rowsplit", "merge", "scalar"):
        gb.spmm(dev(A.rowptr), dev(np.zeros(1, np.int32)), dev(np.zeros(1, np.float32)), dev(B), out=out,
                variant=variant)
        assert torch.all(out == 0)
    # M = 1 and a single column
    A = gen.csr_uniform(1, 500, 0.5, seed=3)
    B = gen.dense_normal(500, 64, 4)
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    for variant in ("rowsplit", "merge"):
        assert_within(run_spmm(gb, A, B, variant=variant), ref, scale, TOL, "M=1")
    # M = 0 is a no-op
    gb.spmm(dev(np.zeros(1, np.int32)), dev(np.zeros(1, np.int32)), dev(np.zeros(1, np.float32)), dev(B))


def test_spmm_plain_entry_point(gb):
    import torch

    A = mat("uniform1024")
    B = gen.dense_normal(A.K, 64, 31)
    C = torch.empty((A.M, 64), device="cuda")
    gb.spmm_csr(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), C, A.M, A.K, 64)
    torch.cuda.synchronize()
    ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C.cpu().numpy(), ref, scale, TOL, "spmm_csr")


def test_spmm_deterministic(gb):
    A = mat("powerlaw")
    B = gen.dense_normal(A.K, 64, 32)
    for variant in ("rowsplit", "merge"):
        c1 = run_spmm(gb, A, B, variant=variant)
        c2 = run_spmm(gb, A, B, variant=variant)
        assert np.array_equal(c1, c2)


# ---- SDDMM --------------------------------------------------------------------------------

def run_sddmm(gb, S, X, Y, **kw):
    return gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(S.vals), dev(X), dev(Y), **kw).cpu().numpy()


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("Kd", [2, 4, 8, 16, 32, 36, 64, 128, 256, 512, 33])
@pytest.mark.parametrize("variant", ["auto", "merge", "entry"])
def test_sddmm_fp32(gb, name, Kd, variant):
    S = mat(name)
    X, Y = gen.dense_normal(S.M, Kd, 41), gen.dense_normal(S.K, Kd, 42)
    if variant != "auto" and Kd % 4:
        with pytest.raises(gb.GbspError, match="ALIGN"):
            run_sddmm(gb, S, X, Y, variant=variant)
        return
    out = run_sddmm(gb, S, X, Y, variant=variant)
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out, ref, scale, TOL, f"{name} Kd={Kd} {variant}")


@pytest.mark.parametrize("vecs", [1, 2, 4])
@pytest.mark.parametrize("Kd", [8, 32, 40, 128, 256, 512])
@pytest.mark.parametrize("variant", ["rowsplit", "merge", "entry"])
def test_sddmm_layouts(gb, vecs, Kd, variant):
    S = mat("powerlaw")
    X, Y = gen.dense_normal(S.M, Kd, 51), gen.dense_normal(S.K, Kd, 52)
    out = run_sddmm(gb, S, X, Y, vecs=vecs, variant=variant)
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out, ref, scale, TOL, f"vecs={vecs} Kd={Kd}")


def _entry_edge_cases():
    """Row-length patterns that stress the entry split's row search: runs of empty rows longer
    than a 32-entry chunk's 32 row ends, single-entry rows, rows of 31 / 32 / 33 entries,
    a long row, and empty rows at both ends."""
    rng = np.random.default_rng(61)
    lengths = np.concatenate([
        np.zeros(70, np.int64), np.ones(100, np.int64), np.zeros(40, np.int64), [31, 32, 33, 1, 0, 64],
        np.zeros(200, np.int64), rng.integers(0, 5, 300), [900], rng.integers(0, 3, 500), np.zeros(37, np.int64)])
    return gen.csr_from_lengths(lengths, 1000, seed=62)


@pytest.mark.parametrize("Kd", [4, 32, 64, 132, 512])
@pytest.mark.parametrize("variant", ["entry", "auto"])
def test_sddmm_entry_split_edge_cases(gb, Kd, variant):
    S = _entry_edge_cases()
    assert S.nnz < 32 * S.M  # auto takes the entry split here
    X, Y = gen.dense_normal(S.M, Kd, 63), gen.dense_normal(S.K, Kd, 64)
    out = run_sddmm(gb, S, X, Y, variant=variant)
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out, ref, scale, TOL, f"entry split Kd={Kd}")


@pytest.mark.parametrize("nnz", [0, 1, 5, 31, 32, 33])
def test_sddmm_entry_split_tiny(gb, nnz):
    import torch

    rng = np.random.default_rng(nnz)
    lengths = np.zeros(50, np.int64)
    lengths[rng.choice(50, nnz, replace=True)] += 1 if nnz else 0
    S = gen.csr_from_lengths(lengths, 60, seed=65)
    X, Y = gen.dense_int(S.M, 32, 66), gen.dense_int(S.K, 32, 67)
    out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(S.vals) if S.nnz else torch.zeros(1, device="cuda"), dev(X),
                   dev(Y), out=torch.full((max(S.nnz, 1),), np.nan, device="cuda"), variant="entry").cpu().numpy()
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    if S.nnz:
        assert_within(out[:S.nnz], ref, scale, TOL, f"entry split nnz={nnz}")


def test_spmm_rejects_entry_split(gb):
    A = mat("ragged")
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        run_spmm(gb, A, gen.dense_normal(A.K, 8, 68), variant="entry")


@pytest.mark.parametrize("Kd", [8, 32, 128])
def test_sddmm_scalar_variant(gb, Kd):
    S = mat("powerlaw")
    X, Y = gen.dense_normal(S.M, Kd, 43), gen.dense_normal(S.K, Kd, 44)
    out = run_sddmm(gb, S, X, Y, variant="scalar")
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out, ref, scale, TOL, f"scalar Kd={Kd}")


@pytest.mark.parametrize("Kd", [2, 32, 128])
def test_sddmm_integers_and_all_ones_mask(gb, Kd):
    M, N = 70, 90
    rp = (np.arange(M + 1) * N).astype(np.int32)
    ci = np.tile(np.arange(N, dtype=np.int32), M)
    S = gen.CSR(M, N, rp, ci, np.ones(M * N, dtype=np.float32))
    X, Y = gen.dense_int(M, Kd, 45), gen.dense_int(N, Kd, 46)
    out = run_sddmm(gb, S, X, Y)
    assert np.array_equal(out.astype(np.int64), (X.astype(np.int64) @ Y.astype(np.int64).T).ravel())


def test_sddmm_plain_entry_point(gb):
    import torch

    S = mat("uniform1024")
    X, Y = gen.dense_normal(S.M, 32, 47), gen.dense_normal(S.K, 32, 48)
    out = torch.empty(S.nnz, device="cuda")
    gb.sddmm_csr(dev(S.rowptr), dev(S.colidx), dev(S.vals), dev(X), dev(Y), out, S.M, S.K, 32)
    torch.cuda.synchronize()
    ref, scale = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out.cpu().numpy(), ref, scale, TOL, "sddmm_csr")


def test_cross_identity_on_gpu(gb):
    """Row sums of SDDMM equal <X_i, (S Y)_i> with both sides computed by the kernels."""
    S = mat("powerlaw")
    X, Y = gen.dense_normal(S.M, 64, 49), gen.dense_normal(S.K, 64, 50)
    out = run_sddmm(gb, S, X, Y).astype(np.float64)
    SY = run_spmm(gb, S, Y).astype(np.float64)
    rows = np.repeat(np.arange(S.M), S.row_lengths())
    lhs = np.bincount(rows, weights=out, minlength=S.M)
    rhs = np.einsum("ik,ik->i", X.astype(np.float64), SY)
    _, sc = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    bound = np.bincount(rows, weights=sc, minlength=S.M)
    assert np.all(np.abs(lhs - rhs) <= 4 * TOL * bound + 1e-30)


# ---- validation ----------------------------------------------------------------------------

def test_validate(gb):
    A = mat("powerlaw")
    assert gb.csr_validate(dev(A.rowptr), dev(A.colidx), A.K) == 0
    bad_ci = A.colidx.copy()
    bad_ci[[3, 10, 500]] = [A.K, -1, A.K + 7]
    assert gb.csr_validate(dev(A.rowptr), dev(bad_ci), A.K) == 3
    bad_rp = A.rowptr.copy()
    bad_rp[5] = bad_rp[6] + 1  # one decrease (rowptr[5] > rowptr[6]); rowptr[4] <= rowptr[5] still
    assert gb.csr_validate(dev(bad_rp), dev(A.colidx), A.K) == 1
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        gb.spmm(dev(A.rowptr), dev(bad_ci), dev(A.vals), dev(gen.dense_normal(A.K, 8, 1)), validate=True)
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        X = dev(gen.dense_normal(A.M, 8, 2))
        gb.sddmm(dev(A.rowptr), dev(bad_ci), dev(A.vals), X, dev(gen.dense_normal(A.K, 8, 3)), validate=True)


# ---- the benchmark's workload, in the benchmark's launch configuration ---------------------

@pytest.fixture(scope="module")
def big():
    return gen.csr_uniform(65536, 65536, 0.99, seed=1001)


def test_spmm_full_size_sampled_rows(gb, big):
    """65,536^2 at 99% (42.9M nnz), N = 64, default launch: 600 sampled rows vs the oracle."""
    A = big
    B = gen.dense_normal(A.K, 64, 1002)
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)).cpu().numpy()
    rows = np.sort(np.random.default_rng(7).choice(A.M, 600, replace=False))
    rows = np.concatenate([[0, A.M - 1], rows])
    rp, ci, v, _ = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    ref, scale = oracle.spmm(rp, ci, v, B)
    assert_within(C[rows], ref, scale, TOL, "full-size spmm")


def test_sddmm_full_size_sampled_rows(gb, big):
    S = big
    X, Y = gen.dense_normal(S.M, 32, 1003), gen.dense_normal(S.K, 32, 1004)
    out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(S.vals), dev(X), dev(Y)).cpu().numpy()
    rows = np.sort(np.random.default_rng(8).choice(S.M, 600, replace=False))
    rp, ci, v, idx = sub_csr(S.rowptr, S.colidx, S.vals, rows)
    ref, scale = oracle.sddmm(rp, ci, v, X[rows], Y)
    assert_within(out[idx], ref, scale, TOL, "full-size sddmm")


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_paired_default_layout_matches_strided_bitwise(gb, dt):
    """For 128-byte rows with 32-byte aligned B the default layout fetches each lane's two
    vectors with one 32-byte load; the strided layout with two vectors per lane has the same
    lane groups and per-column order, so the two give the same bits (the merge path with the
    same grid: its default grid follows each kernel's occupancy, and the split of the merge
    path sets where carries are added)."""
    A = gen.csr_powerlaw(3000, 2500, 0.99, seed=781)
    N = 32 if dt == "f32" else 64
    B = gen.dense_normal(A.K, N, 782)
    rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
    if dt == "bf16":
        v, Bd = gb.quantize_bf16(v), gb.quantize_bf16(Bd)
    for variant, cps in (("rowsplit", 0), ("merge", 2)):
        paired = gb.spmm(rp, ci, v, Bd, variant=variant, ctas_per_sm=cps).cpu().numpy()
        strided = gb.spmm(rp, ci, v, Bd, variant=variant, ctas_per_sm=cps, vecs=2).cpu().numpy()
        assert np.array_equal(paired, strided)


@pytest.mark.parametrize("Kd", [32, 64, 128])
def test_sddmm_16_byte_aligned_operands_take_the_one_vector_layout(gb, Kd):
    """X and Y rows 16-byte but not 32-byte aligned cannot take the paired 32-byte loads;
    the one-vector layout must give the oracle's result just the same."""
    import torch

    A = gen.csr_powerlaw(2000, 1500, 0.99, seed=791)
    X, Y = gen.dense_normal(A.M, Kd, 792), gen.dense_normal(A.K, Kd, 793)
    Xb = torch.zeros(A.M * Kd + 4, device="cuda")
    Yb = torch.zeros(A.K * Kd + 4, device="cuda")
    Xd = Xb[4:].view(A.M, Kd)  # 16 bytes past a 256-byte boundary
    Yd = Yb[4:].view(A.K, Kd)
    Xd.copy_(dev(X))
    Yd.copy_(dev(Y))
    assert Xd.data_ptr() % 32 == 16 and Yd.data_ptr() % 32 == 16
    out = gb.sddmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), Xd, Yd).cpu().numpy()
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, X, Y)
    assert_within(out, ref, sc, TOL, f"sddmm one-vector layout Kd={Kd}")


@pytest.mark.parametrize("variant", ["rowsplit", "merge"])
def test_spmm_128_byte_rows_16_byte_aligned_b(gb, variant):
    """FP32 N = 32 with B 16-byte but not 32-byte aligned: the strided layout instead of
    the paired one, same result as the oracle."""
    import torch

    A = gen.csr_powerlaw(2000, 1500, 0.99, seed=794)
    B = gen.dense_normal(A.K, 32, 795)
    Bb = torch.zeros(A.K * 32 + 4, device="cuda")
    Bd = Bb[4:].view(A.K, 32)
    Bd.copy_(dev(B))
    assert Bd.data_ptr() % 32 == 16
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), Bd, variant=variant).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL, f"spmm strided 128-byte rows {variant}")

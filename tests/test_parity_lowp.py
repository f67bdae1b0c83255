"""GPU parity of the BF16 and per-row-scaled FP8-E4M3 forms (FP32 accumulation).

Two checks per form:
  * against the FP64 oracle run on the dequantised operands (the oracle's own rounding,
    which the first tests show is bit-identical to the library's): isolates the kernel
    arithmetic, FP32 tolerance |err| <= 1e-5 * scale;
  * against the FP64 oracle on the original FP32 operands (quantisation included):
    |err| <= 1e-2 * scale for BF16 and <= 4e-2 * scale for E4M3.
Roundings themselves are integer (byte) results and must match the oracle bit for bit.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu
TOL32, TOL_BF16, TOL_E4M3 = 1e-5, 1e-2, 4e-2


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def _bits(t):
    import torch

    return t.view(torch.int16).cpu().numpy().view(np.uint16) if t.dtype == torch.bfloat16 else t.cpu().numpy()


# ---- roundings: bit-exact --------------------------------------------------------------------

def test_bf16_rounding_bit_exact(gb):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32),
                        rng.integers(0, 2**32, 100000, dtype=np.uint64).astype(np.uint32).view(np.float32),
                        np.array([0.0, -0.0, 1.0 + 2**-8, 3e38, -3e38, 1e-40], dtype=np.float32)])
    x = x[np.isfinite(x)]
    assert np.array_equal(_bits(gb.quantize_bf16(dev(x))), oracle.bf16_round(x))


@pytest.mark.parametrize("shape", [(300, 64), (17, 256), (1, 5)])
def test_e4m3_dense_rows_bit_exact(gb, shape):
    x = gen.dense_normal(*shape, seed=2) * np.float32(3.0)
    x[0, :] = 0.0  # an all-zero row gets scale 1
    q, s = gb.quantize_e4m3_rows(dev(x))
    qo, so = oracle.e4m3_rows(x)
    assert np.array_equal(q.cpu().numpy(), qo)
    assert np.array_equal(s.cpu().numpy(), so)


def test_e4m3_csr_rows_bit_exact(gb):
    A = gen.csr_powerlaw(4000, 3000, 0.99, seed=3)
    q, s = gb.quantize_e4m3_rows(dev(A.vals), dev(A.rowptr))
    qo, so = oracle.e4m3_rows(A.vals, A.rowptr)
    assert np.array_equal(q.cpu().numpy(), qo)
    assert np.array_equal(s.cpu().numpy(), so)


# ---- SpMM ------------------------------------------------------------------------------------

def _spmm_bf16(gb, A, B, **kw):
    qa, qb = gb.quantize_bf16(dev(A.vals)), gb.quantize_bf16(dev(B))
    return gb.spmm(dev(A.rowptr), dev(A.colidx), qa, qb, **kw).cpu().numpy()


def _spmm_e4m3(gb, A, B, **kw):
    qa, sa = gb.quantize_e4m3_rows(dev(A.vals), dev(A.rowptr))
    qb, tb = gb.quantize_e4m3_rows(dev(B))
    return gb.spmm(dev(A.rowptr), dev(A.colidx), qa, qb, a_scale=sa, b_scale=tb, **kw).cpu().numpy()


STRUCTS = {
    "uniform": lambda: gen.csr_uniform(2048, 2048, 0.9, seed=11),
    "clustered": lambda: gen.csr_clustered(2048, 2048, 0.9, seed=12),
    "powerlaw": lambda: gen.csr_powerlaw(3000, 2000, 0.98, seed=13),
}
_cache = {}


def mat(k):
    if k not in _cache:
        _cache[k] = STRUCTS[k]()
    return _cache[k]


@pytest.mark.parametrize("struct", list(STRUCTS))
@pytest.mark.parametrize("N", [64, 256, 136])
@pytest.mark.parametrize("variant", ["rowsplit", "merge"])
@pytest.mark.parametrize("vecs", [1, 2])
def test_spmm_bf16(gb, struct, N, variant, vecs):
    A = mat(struct)
    B = gen.dense_normal(A.K, N, 14)
    C = _spmm_bf16(gb, A, B, variant=variant, vecs=vecs)
    da = oracle.bf16_decode(oracle.bf16_round(A.vals))
    db = oracle.bf16_decode(oracle.bf16_round(B))
    ref, sc = oracle.spmm(A.rowptr, A.colidx, da, db)
    assert_within(C, ref, sc, TOL32, f"bf16 dequantised {struct} N={N}")
    ref0, sc0 = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref0, sc0, TOL_BF16, f"bf16 vs fp32 {struct} N={N}")


@pytest.mark.parametrize("struct", list(STRUCTS))
@pytest.mark.parametrize("N", [64, 256, 144])
@pytest.mark.parametrize("variant", ["rowsplit", "merge"])
def test_spmm_e4m3(gb, struct, N, variant):
    A = mat(struct)
    B = gen.dense_normal(A.K, N, 15)
    C = _spmm_e4m3(gb, A, B, variant=variant)
    qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    qb, tb = oracle.e4m3_rows(B)
    ref, sc = oracle.spmm(A.rowptr, A.colidx, oracle.e4m3_rows_dequant(qa, sa, A.rowptr),
                          oracle.e4m3_rows_dequant(qb, tb))
    assert_within(C, ref, sc, TOL32, f"e4m3 dequantised {struct} N={N}")
    if struct != "powerlaw":  # rows of a few entries need not meet the 4e-2 quantisation bound
        ref0, sc0 = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
        assert_within(C, ref0, sc0, TOL_E4M3, f"e4m3 vs fp32 {struct} N={N}")


def test_spmm_lowp_scalar_widths(gb):
    A = mat("powerlaw")
    for N in (5, 24):
        B = gen.dense_normal(A.K, N, 16)
        C = _spmm_bf16(gb, A, B)
        da = oracle.bf16_decode(oracle.bf16_round(A.vals))
        ref, sc = oracle.spmm(A.rowptr, A.colidx, da, oracle.bf16_decode(oracle.bf16_round(B)))
        assert_within(C, ref, sc, TOL32, f"bf16 scalar N={N}")
        C = _spmm_e4m3(gb, A, B)
        qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
        qb, tb = oracle.e4m3_rows(B)
        ref, sc = oracle.spmm(A.rowptr, A.colidx, oracle.e4m3_rows_dequant(qa, sa, A.rowptr),
                              oracle.e4m3_rows_dequant(qb, tb))
        assert_within(C, ref, sc, TOL32, f"e4m3 scalar N={N}")


@pytest.mark.parametrize("variant", ["rowsplit", "merge", "scalar"])
def test_spmm_lowp_integers_bit_exact(gb, variant):
    """Integers in [-8, 8] are exact in BF16 and in E4M3 with unit scales."""
    import torch

    A = gen.csr_powerlaw(1500, 1200, 0.97, seed=17)
    vals = gen.vals_int(A.nnz, 18)
    B = gen.dense_int(A.K, 64, 19)
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(oracle.bf16_round(vals).view(np.int16)).view(torch.bfloat16),
                dev(oracle.bf16_round(B).view(np.int16)).view(torch.bfloat16), variant=variant).cpu().numpy()
    assert np.array_equal(C.astype(np.float64), want)
    ones_m, ones_k = dev(np.ones(A.M, np.float32)), dev(np.ones(A.K, np.float32))
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(oracle.e4m3_round(vals)), dev(oracle.e4m3_round(B)),
                a_scale=ones_m, b_scale=ones_k, variant=variant).cpu().numpy()
    assert np.array_equal(C.astype(np.float64), want)


# ---- SDDMM -----------------------------------------------------------------------------------

@pytest.mark.parametrize("Kd", [32, 128, 256, 40])
@pytest.mark.parametrize("variant", ["rowsplit", "merge", "entry"])
def test_sddmm_bf16(gb, Kd, variant):
    S = mat("uniform")
    X, Y = gen.dense_normal(S.M, Kd, 21), gen.dense_normal(S.K, Kd, 22)
    out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(S.vals), gb.quantize_bf16(dev(X)),
                   gb.quantize_bf16(dev(Y)), variant=variant).cpu().numpy()
    dx, dy = oracle.bf16_decode(oracle.bf16_round(X)), oracle.bf16_decode(oracle.bf16_round(Y))
    ref, sc = oracle.sddmm(S.rowptr, S.colidx, S.vals, dx, dy)
    assert_within(out, ref, sc, TOL32, f"bf16 dequantised Kd={Kd}")
    ref0, sc0 = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    assert_within(out, ref0, sc0, TOL_BF16, f"bf16 vs fp32 Kd={Kd}")


@pytest.mark.parametrize("Kd", [32, 128, 256, 48])
@pytest.mark.parametrize("variant", ["rowsplit", "merge", "entry"])
def test_sddmm_e4m3(gb, Kd, variant):
    S = mat("clustered")
    X, Y = gen.dense_normal(S.M, Kd, 23), gen.dense_normal(S.K, Kd, 24)
    qx, u = gb.quantize_e4m3_rows(dev(X))
    qy, w = gb.quantize_e4m3_rows(dev(Y))
    out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(S.vals), qx, qy, x_scale=u, y_scale=w,
                   variant=variant).cpu().numpy()
    oqx, ou = oracle.e4m3_rows(X)
    oqy, ow = oracle.e4m3_rows(Y)
    ref, sc = oracle.sddmm(S.rowptr, S.colidx, S.vals, oracle.e4m3_rows_dequant(oqx, ou),
                           oracle.e4m3_rows_dequant(oqy, ow))
    assert_within(out, ref, sc, TOL32, f"e4m3 dequantised Kd={Kd}")
    ref0, sc0 = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    if Kd >= 128:
        # the E4M3 configuration's width (Kd = 256): every output within 4e-2 of its scale
        assert_within(out, ref0, sc0, TOL_E4M3, f"e4m3 vs fp32 Kd={Kd}")
    else:
        # a narrow dot product averages few rounding errors: with E4M3's 2^-4 relative
        # step the largest of ~2M outputs can pass 4e-2 (about 0.057 / sqrt(Kd) per
        # standard deviation), so only the mean is bounded here
        rel = np.abs(out - ref0)[sc0 > 0] / sc0[sc0 > 0]
        assert rel.mean() <= TOL_E4M3 / 4


def test_sddmm_lowp_integers_bit_exact(gb):
    import torch

    S = mat("powerlaw")
    X, Y = gen.dense_int(S.M, 64, 25), gen.dense_int(S.K, 64, 26)
    svals = gen.vals_int(S.nnz, 27)
    want, _ = oracle.sddmm(S.rowptr, S.colidx, svals, X, Y)
    out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(svals), dev(oracle.bf16_round(X).view(np.int16)).view(torch.bfloat16),
                   dev(oracle.bf16_round(Y).view(np.int16)).view(torch.bfloat16)).cpu().numpy()
    assert np.array_equal(out.astype(np.float64), want)
    for variant in ("auto", "entry"):
        out = gb.sddmm(dev(S.rowptr), dev(S.colidx), dev(svals), dev(oracle.e4m3_round(X)), dev(oracle.e4m3_round(Y)),
                       x_scale=dev(np.ones(S.M, np.float32)), y_scale=dev(np.ones(S.K, np.float32)),
                       variant=variant).cpu().numpy()
        assert np.array_equal(out.astype(np.float64), want)


# ---- every E4M3 code: the gathered operand's decode ------------------------------------------

def _finite_codes():
    """The 254 finite E4M3 codes (0x7F and 0xFF are NaN), then +0 and -0 again: 256 columns."""
    c = np.array([q for q in range(256) if q & 0x7F != 0x7F] + [0x00, 0x80], dtype=np.uint8)
    assert c.size == 256
    return c


@pytest.mark.parametrize("variant", ["rowsplit", "merge", "rowgroup", "scalar"])
@pytest.mark.parametrize("t", [1.0, 2.0**-40, 2.0**50])
def test_spmm_e4m3_every_code_exact(gb, variant, t):
    """C = A B with one entry of value 1 per row (C's rows are B's rows): every finite code,
    subnormals included, decodes to exactly the oracle's value times the row scale t."""
    codes = _finite_codes()
    K = 256
    B = np.stack([np.roll(codes, k) for k in range(K)])            # every code in every column
    rowptr = np.arange(K + 1, dtype=np.int32)
    colidx = np.arange(K, dtype=np.int32)
    one = oracle.e4m3_round(np.ones(K, np.float32))
    C = gb.spmm(dev(rowptr), dev(colidx), dev(one), dev(B), a_scale=dev(np.ones(K, np.float32)),
                b_scale=dev(np.full(K, t, np.float32)), variant=variant).cpu().numpy()
    want = oracle.e4m3_decode(B) * t
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("variant", ["rowsplit", "merge", "entry", "scalar"])
def test_sddmm_e4m3_every_code_exact(gb, variant):
    """out_ij = s_ij <X_i, Y_j> with X_i the unit vector e_i: every finite code of Y read exactly."""
    codes = _finite_codes()
    M, Nr, Kd = 256, 64, 256
    X = np.zeros((M, Kd), np.float32)
    X[np.arange(M), np.arange(M)] = 1.0
    Y = np.stack([np.roll(codes, 4 * j) for j in range(Nr)])
    rowptr = (np.arange(M + 1) * Nr).astype(np.int32)
    colidx = np.tile(np.arange(Nr, dtype=np.int32), M)
    svals = np.where(np.arange(M * Nr) % 3 == 0, -0.5, 2.0).astype(np.float32)
    out = gb.sddmm(dev(rowptr), dev(colidx), dev(svals), dev(oracle.e4m3_round(X)), dev(Y),
                   x_scale=dev(np.ones(M, np.float32)), y_scale=dev(np.ones(Nr, np.float32)),
                   variant=variant).cpu().numpy()
    rows = np.repeat(np.arange(M), Nr)
    want = svals.astype(np.float64) * oracle.e4m3_decode(Y)[colidx, rows]
    assert np.array_equal(out.astype(np.float64), want)

"""Pins for the FP64 oracle: each check comes from outside the oracle itself (brute force,
library routines, closed forms, invariants, the paper's printed numbers)."""
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_csr(M, K, density, seed, dup=False, shuffle=False):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(M):
        L = rng.binomial(K, density)
        c = list(rng.choice(K, L, replace=False)) if L else []
        if dup and c:
            c = c + [c[0]]
        if shuffle:
            rng.shuffle(c)
        rows += [i] * len(c)
        cols += c
    vals = rng.uniform(-1, 1, len(cols))
    rowptr = np.zeros(M + 1, dtype=np.int32)
    np.add.at(rowptr, np.asarray(rows, dtype=np.int64) + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), np.asarray(cols, dtype=np.int32), vals


def _dense(rowptr, colidx, vals, K):
    M = len(rowptr) - 1
    A = np.zeros((M, K))
    for i in range(M):
        for p in range(rowptr[i], rowptr[i + 1]):
            A[i, colidx[p]] += vals[p]
    return A


def test_worked_example():
    """Hand-computed terms of Eq. 1 and Eq. 2 (tests/golden/spmm_sddmm_worked_3x4.txt)."""
    d = {}
    for line in open(os.path.join(GOLDEN, "spmm_sddmm_worked_3x4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = np.array([float(t) for t in v])
    rp, ci = d["rowptr"].astype(np.int32), d["colidx"].astype(np.int32)
    C, _ = oracle.spmm(rp, ci, d["vals"], d["B"].reshape(4, 2))
    np.testing.assert_array_equal(C.ravel(), d["C"])
    out, _ = oracle.sddmm(rp, ci, d["vals"], d["X"].reshape(3, 2), d["Y"].reshape(4, 2))
    np.testing.assert_array_equal(out, d["out"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spmm_brute_force_tiny(seed):
    """Triple loop over a densified A, in plain Python floats, with repeated and unsorted
    column indices and empty rows."""
    rng = np.random.default_rng(100 + seed)
    M, K, N = int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(1, 6))
    rp, ci, v = _rand_csr(M, K, 0.4, seed, dup=True, shuffle=True)
    B = rng.standard_normal((K, N))
    A = _dense(rp, ci, v, K)
    ref = [[sum(A[i][k] * B[k][n] for k in range(K)) for n in range(N)] for i in range(M)]
    C, S = oracle.spmm(rp, ci, v, B)
    np.testing.assert_allclose(C, np.array(ref).reshape(M, N), rtol=1e-12, atol=1e-12)
    sref = np.zeros((M, N))
    for i in range(M):
        for p in range(rp[i], rp[i + 1]):
            sref[i] += abs(v[p]) * np.abs(B[ci[p]])
    np.testing.assert_allclose(S, sref, rtol=1e-12, atol=1e-14)


def test_spmm_matches_numpy_matmul():
    rp, ci, v = _rand_csr(120, 90, 0.1, 7, dup=True, shuffle=True)
    B = np.random.default_rng(8).standard_normal((90, 33))
    A = _dense(rp, ci, v, 90)
    C, S = oracle.spmm(rp, ci, v, B)
    np.testing.assert_allclose(C, A @ B, rtol=1e-11, atol=1e-12)
    # the scale of a matrix without repeats is |A| |B|
    rp2, ci2, v2 = _rand_csr(60, 50, 0.2, 9)
    _, S2 = oracle.spmm(rp2, ci2, v2, B[:50])
    np.testing.assert_allclose(S2, np.abs(_dense(rp2, ci2, v2, 50)) @ np.abs(B[:50]), rtol=1e-12)


def test_spmm_identity_returns_b_exactly():
    K = 64
    rp = np.arange(K + 1, dtype=np.int32)
    ci = np.arange(K, dtype=np.int32)
    B = gen.dense_normal(K, 24, 3).astype(np.float64)
    C, _ = oracle.spmm(rp, ci, np.ones(K), B)
    assert np.array_equal(C, B)


def test_spmm_exact_integers():
    A = gen.csr_uniform(256, 192, 0.9, seed=11)
    vals = gen.vals_int(A.nnz, 12)
    B = gen.dense_int(192, 40, 13)
    C, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    Ad = np.zeros((256, 192), dtype=np.int64)
    for i in range(256):
        Ad[i, A.colidx[A.rowptr[i]:A.rowptr[i + 1]]] = vals[A.rowptr[i]:A.rowptr[i + 1]].astype(np.int64)
    assert np.array_equal(C, (Ad @ B.astype(np.int64)).astype(np.float64))


def test_spmm_linearity():
    A = gen.csr_uniform(200, 150, 0.95, seed=21)
    B1, B2 = gen.dense_normal(150, 16, 22), gen.dense_normal(150, 16, 23)
    a, b = 0.75, -2.5
    C12, _ = oracle.spmm(A.rowptr, A.colidx, A.vals, a * B1.astype(np.float64) + b * B2.astype(np.float64))
    C1, _ = oracle.spmm(A.rowptr, A.colidx, A.vals, B1)
    C2, _ = oracle.spmm(A.rowptr, A.colidx, A.vals, B2)
    np.testing.assert_allclose(C12, a * C1 + b * C2, rtol=1e-12, atol=1e-12)


def test_spmm_empty_rows_and_no_entries():
    rp = np.zeros(6, dtype=np.int32)
    C, S = oracle.spmm(rp, np.zeros(0, np.int32), np.zeros(0), np.ones((4, 3)))
    assert C.shape == (5, 3) and not C.any() and not S.any()
    rp = np.array([0, 0, 2, 2], dtype=np.int32)
    C, _ = oracle.spmm(rp, np.array([0, 1], np.int32), np.array([1.0, 1.0]), np.eye(2))
    np.testing.assert_array_equal(C, [[0, 0], [1, 1], [0, 0]])


def test_spmm_permutation_within_rows():
    A = gen.csr_uniform(64, 512, 0.8, seed=31)
    B = gen.dense_normal(512, 8, 32)
    rng = np.random.default_rng(33)
    ci, v = A.colidx.copy(), A.vals.copy()
    for i in range(64):
        s, e = A.rowptr[i], A.rowptr[i + 1]
        perm = rng.permutation(e - s)
        ci[s:e], v[s:e] = ci[s:e][perm], v[s:e][perm]
    C1, _ = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    C2, _ = oracle.spmm(A.rowptr, ci, v, B)
    np.testing.assert_allclose(C1, C2, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_sddmm_brute_force_tiny(seed):
    rng = np.random.default_rng(200 + seed)
    M, N, Kd = int(rng.integers(1, 8)), int(rng.integers(1, 8)), int(rng.integers(1, 6))
    rp, ci, s = _rand_csr(M, N, 0.5, seed + 40, dup=True, shuffle=True)
    X, Y = rng.standard_normal((M, Kd)), rng.standard_normal((N, Kd))
    ref = []
    for i in range(M):
        for p in range(rp[i], rp[i + 1]):
            ref.append(s[p] * sum(X[i][k] * Y[ci[p]][k] for k in range(Kd)))
    out, S = oracle.sddmm(rp, ci, s, X, Y)
    np.testing.assert_allclose(out, np.array(ref), rtol=1e-12, atol=1e-12)
    sref = [abs(s[p]) * float(np.abs(X[i]) @ np.abs(Y[ci[p]])) for i in range(M) for p in range(rp[i], rp[i + 1])]
    np.testing.assert_allclose(S, np.array(sref), rtol=1e-12, atol=1e-14)


def test_sddmm_all_ones_mask_gives_x_yt():
    """An all-ones S on the full pattern returns exactly the entries of X Y^T (M != N)."""
    M, N, Kd = 13, 21, 7
    X = gen.dense_int(M, Kd, 1)
    Y = gen.dense_int(N, Kd, 2)
    rp = (np.arange(M + 1) * N).astype(np.int32)
    ci = np.tile(np.arange(N, dtype=np.int32), M)
    out, _ = oracle.sddmm(rp, ci, np.ones(M * N), X, Y)
    assert np.array_equal(out, (X.astype(np.int64) @ Y.astype(np.int64).T).ravel().astype(np.float64))
    Xn, Yn = gen.dense_normal(M, Kd, 3), gen.dense_normal(N, Kd, 4)
    out, _ = oracle.sddmm(rp, ci, np.ones(M * N), Xn, Yn)
    np.testing.assert_allclose(out, (Xn.astype(np.float64) @ Yn.astype(np.float64).T).ravel(), rtol=1e-12, atol=1e-12)


def test_sddmm_multiplies_by_s_values():
    """Eq. 2 multiplies by the values of S (not a 0/1 mask): out(S) = s * out(pattern)."""
    S = gen.csr_uniform(50, 70, 0.8, seed=51)
    X, Y = gen.dense_normal(50, 9, 52), gen.dense_normal(70, 9, 53)
    o1, _ = oracle.sddmm(S.rowptr, S.colidx, np.ones(S.nnz), X, Y)
    os_, _ = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    np.testing.assert_array_equal(os_, S.vals.astype(np.float64) * o1)
    full = X.astype(np.float64) @ Y.astype(np.float64).T
    rows = np.repeat(np.arange(50), S.row_lengths())
    np.testing.assert_allclose(o1, full[rows, S.colidx], rtol=1e-12, atol=1e-12)


def test_cross_identity_sddmm_rowsum_equals_x_dot_spmm():
    """sum over row i of sddmm(S, X, Y) = <X_i, (S Y)_i>: ties Eq. 1 and Eq. 2 together."""
    S = gen.csr_powerlaw(300, 200, 0.9, seed=61)
    X, Y = gen.dense_normal(300, 12, 62), gen.dense_normal(200, 12, 63)
    out, _ = oracle.sddmm(S.rowptr, S.colidx, S.vals, X, Y)
    SY, _ = oracle.spmm(S.rowptr, S.colidx, S.vals, Y)
    rows = np.repeat(np.arange(300), S.row_lengths())
    lhs = np.bincount(rows, weights=out, minlength=300)
    rhs = np.einsum("ik,ik->i", X.astype(np.float64), SY)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-10)


def test_footprint_pin():
    """Section V-B: N = 262144 at 1e-4 density, CSR about 53 MB, dense FP32 256 GB."""
    g = json.load(open(os.path.join(GOLDEN, "footprint_n262144.json")))
    n = g["n"]
    nnz = gen.nnz_for(n, n, density=g["density"])
    assert nnz == 6_871_948
    csr_bytes = 8 * nnz + 4 * (n + 1)
    assert abs(csr_bytes / 2**20 - g["csr_mib_approx"]) <= g["csr_rel_tol"] * g["csr_mib_approx"]
    assert 4 * n * n == g["dense_gib"] * 2**30


# ---- BF16 / E4M3 roundings ------------------------------------------------------------

def test_bf16_round_pins():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, 1.0 + 2**-8 + 2**-20, -2.5, 0.0, -0.0,
                  3.0e38, np.inf, -np.inf], dtype=np.float32)
    # 1+2^-8 is half an ulp above 1 -> ties to the even pattern 0x3F80; 1+3*2^-8 is half
    # way between 0x3F81 (odd) and 0x3F82 (even) -> 0x3F82; just above half rounds up.
    want = np.array([0x3F80, 0x3F80, 0x3F82, 0x3F81, 0xC020, 0x0000, 0x8000, 0x7F62, 0x7F80,
                     0xFF80], dtype=np.uint16)
    assert np.array_equal(oracle.bf16_round(x), want)
    assert np.isnan(oracle.bf16_decode(oracle.bf16_round(np.array([np.nan], np.float32))))[0]


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(200000).astype(np.float32),
                        (rng.standard_normal(20000) * 1e-38).astype(np.float32),
                        rng.integers(0, 2**32, 100000, dtype=np.uint64).astype(np.uint32).view(np.float32)])
    x = x[np.isfinite(x)]
    ours = oracle.bf16_round(x)
    theirs = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, theirs)
    np.testing.assert_array_equal(oracle.bf16_decode(ours), torch.from_numpy(x).to(torch.bfloat16).double().numpy())


def test_e4m3_pins():
    x = np.array([0.0, 1.0, -1.0, 448.0, 500.0, -1e9, 2.0**-9, 2.0**-6, 1.0625, 1.1875, 2.0**-10,
                  3 * 2.0**-10, 0.875 * 2**-6], dtype=np.float32)
    want = np.array([0x00, 0x38, 0xB8, 0x7E, 0x7E, 0xFE, 0x01, 0x08, 0x38, 0x3A, 0x00, 0x02, 0x07],
                    dtype=np.uint8)
    assert np.array_equal(oracle.e4m3_round(x), want)
    v = oracle.e4m3_decode(np.arange(256, dtype=np.uint8))
    assert v[0x7E] == 448.0 and v[0x01] == 2.0**-9 and v[0x08] == 2.0**-6 and v[0x38] == 1.0
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    finite = np.isfinite(v)
    assert finite.sum() == 254
    # every finite code survives a round trip
    codes = np.arange(256, dtype=np.uint8)[finite]
    assert np.array_equal(oracle.e4m3_round(v[finite].astype(np.float32)), codes)


def test_e4m3_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    v = oracle.e4m3_decode(np.arange(256, dtype=np.uint8))
    t = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn).double().numpy()
    fin = np.isfinite(v)
    np.testing.assert_array_equal(v[fin], t[fin])
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.uniform(-448, 448, 200000), rng.standard_normal(100000) * 0.01,
                        # midpoints between neighbouring codes: ties must go to even
                        0.5 * (np.sort(v[fin])[1:] + np.sort(v[fin])[:-1])]).astype(np.float32)
    ours = oracle.e4m3_round(x)
    theirs = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, theirs)


def test_e4m3_rows_scale_and_max():
    A = gen.csr_powerlaw(500, 400, 0.9, seed=71)
    q, s = oracle.e4m3_rows(A.vals, A.rowptr)
    for i in range(500):
        seg = A.vals[A.rowptr[i]:A.rowptr[i + 1]]
        if seg.size == 0:
            assert s[i] == 1.0
            continue
        amax = np.float32(np.abs(seg).max())
        assert s[i] == np.float32(amax / np.float32(448.0))
        assert np.abs(oracle.e4m3_decode(q[A.rowptr[i]:A.rowptr[i + 1]])).max() == 448.0
    deq = oracle.e4m3_rows_dequant(q, s, A.rowptr)
    # relative rounding error of E4M3 normals is at most 2^-4
    big = np.abs(A.vals) > np.repeat(s, A.row_lengths()) * 2**-6
    assert np.all(np.abs(deq[big] - A.vals[big]) <= 2**-4 * np.abs(A.vals[big]) * (1 + 1e-6))
    X = gen.dense_normal(30, 64, 72)
    qd, sd = oracle.e4m3_rows(X)
    assert qd.shape == X.shape and sd.shape == (30,)
    np.testing.assert_array_equal(sd, (np.abs(X).max(axis=1) / np.float32(448)).astype(np.float32))


# ---- GAT-style chain: row softmax between SDDMM and SpMM --------------------------------------

def test_row_softmax_hand_example():
    """exp of [0, ln 2, ln 5] is [1, 2, 5]: weights 1/8, 2/8, 5/8; an empty row; equal scores
    split evenly; huge scores do not overflow (the row maximum is subtracted first)."""
    rp = np.array([0, 3, 3, 5, 7])
    E = np.array([0.0, np.log(2.0), np.log(5.0), 10.0, 10.0, 1000.0, 999.0])
    a = oracle.row_softmax(rp, E)
    assert np.allclose(a[:3], [1 / 8, 2 / 8, 5 / 8], rtol=0, atol=1e-15)
    assert np.allclose(a[3:5], [0.5, 0.5], rtol=0, atol=1e-15)
    e = np.exp(-1.0)
    assert np.allclose(a[5:7], [1 / (1 + e), e / (1 + e)], rtol=0, atol=1e-15)


def test_gat_chain_against_dense_brute_force():
    """alpha and O from the chain equal a dense masked softmax (entries outside the pattern at
    -inf) followed by a dense product, written out with plain loops."""
    rng = np.random.default_rng(5)
    n, N = 9, 4
    lengths = rng.integers(0, 5, n)
    A = gen.csr_from_lengths(lengths, n, seed=6)
    H = rng.normal(size=(n, N))
    alpha, O, _ = oracle.gat_chain(A.rowptr, A.colidx, A.vals, H)
    for i in range(n):
        a, b = A.rowptr[i], A.rowptr[i + 1]
        scores = np.full(n, -np.inf)
        for p in range(a, b):
            scores[A.colidx[p]] = A.vals[p] * sum(H[i, k] * H[A.colidx[p], k] for k in range(N))
        if a == b:
            assert np.all(O[i] == 0)
            continue
        w = np.exp(scores - scores.max())
        w = w / w.sum()
        for p in range(a, b):
            assert abs(alpha[p] - w[A.colidx[p]]) <= 1e-14
        for k in range(N):
            assert abs(O[i, k] - sum(w[j] * H[j, k] for j in range(n))) <= 1e-12


def test_gat_chain_invariants():
    """Rows of alpha sum to 1 and are positive; with every H row equal to v, O_i = v on
    non-empty rows (a convex combination of equal vectors)."""
    A = gen.gnn_graph(300, 21)
    H = gen.dense_normal(A.M, 16, 22).astype(np.float64)
    alpha, _, _ = oracle.gat_chain(A.rowptr, A.colidx, A.vals, H)
    sums = np.add.reduceat(alpha, A.rowptr[:-1][A.row_lengths() > 0])
    assert np.allclose(sums, 1.0, rtol=0, atol=1e-12) and np.all(alpha > 0)
    v = np.linspace(-1, 1, 16)
    Hc = np.tile(v, (A.M, 1))
    _, O, _ = oracle.gat_chain(A.rowptr, A.colidx, A.vals, Hc)
    nz = A.row_lengths() > 0
    assert np.allclose(O[nz], v, rtol=0, atol=1e-12) and np.all(O[~nz] == 0)

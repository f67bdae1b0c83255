"""GPU parity of the row-group SpMM variant and of the automatic work split (AUTO).

The row groups give one lane group per row (several rows per warp); AUTO picks the row
split, the merge path or the row groups from the pattern's row lengths, measured once per
pattern.  Integer inputs must match the FP64 oracle bit for bit, random FP32 inputs within
1e-5 of sum |a||b|; the row statistics behind the choice are integers and must equal the
ones counted on the host.
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
    """Half the rows empty, most others 1-6 entries, a few of 40-300."""
    rng = np.random.default_rng(seed)
    kind = rng.random(M)
    lengths = np.zeros(M, np.int64)
    short = (kind >= 0.5) & (kind < 0.97)
    lengths[short] = rng.integers(1, 7, M)[short]
    lengths[kind >= 0.97] = rng.integers(40, 301, M)[kind >= 0.97]
    return lengths


@pytest.mark.parametrize("N", [4, 8, 32, 64, 128, 200, 516])
def test_rowgroup_integers_bit_exact(gb, N):
    A = gen.csr_from_lengths(mixed_lengths(5003, N), 4000, seed=601 + N)
    vals = gen.vals_int(A.nnz, 602)
    B = gen.dense_int(A.K, N, 603)
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(vals), dev(B), variant="rowgroup").cpu().numpy()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("vecs,unroll", [(0, 0), (1, 1), (1, 4), (2, 2), (4, 4)])
def test_rowgroup_random_fp32_layouts(gb, vecs, unroll):
    A = gen.csr_powerlaw(6000, 5000, 0.999, seed=604)
    B = gen.dense_normal(A.K, 128, 605)
    C = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), variant="rowgroup", vecs=vecs,
                unroll=unroll).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL32, f"rowgroup vecs={vecs} unroll={unroll}")


def test_rowgroup_low_precision_forms(gb):
    """BF16 and per-row-scaled E4M3 through the row groups, against the oracle on the
    dequantised operands (the kernel arithmetic, FP32 tolerance)."""
    A = gen.csr_from_lengths(mixed_lengths(3000, 7), 2500, seed=606)
    B = gen.dense_normal(A.K, 96, 607)
    rp, ci = dev(A.rowptr), dev(A.colidx)
    qa, qb = gb.quantize_bf16(dev(A.vals)), gb.quantize_bf16(dev(B))
    C = gb.spmm(rp, ci, qa, qb, variant="rowgroup").cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, oracle.bf16_decode(oracle.bf16_round(A.vals)),
                          oracle.bf16_decode(oracle.bf16_round(B)))
    assert_within(C, ref, sc, TOL32, "rowgroup bf16")
    ea, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    eb, tb = oracle.e4m3_rows(B)
    C8 = gb.spmm(rp, ci, dev(ea), dev(eb), a_scale=dev(sa), b_scale=dev(tb), variant="rowgroup").cpu().numpy()
    ref8, sc8 = oracle.spmm(A.rowptr, A.colidx, oracle.e4m3_rows_dequant(ea, sa, A.rowptr),
                            oracle.e4m3_rows_dequant(eb, tb))
    assert_within(C8, ref8, sc8, TOL32, "rowgroup e4m3")


def test_rowgroup_padded_ld_and_no_rows(gb):
    import torch

    A = gen.csr_from_lengths(mixed_lengths(700, 8), 600, seed=608)
    vals = gen.vals_int(A.nnz, 609)
    B = gen.dense_int(A.K, 72, 610)
    Bp = torch.zeros((A.K, 80), device="cuda")
    Bp[:, :64] = dev(B[:, :64])
    Cp = torch.full((A.M, 68), 7.0, device="cuda")
    gb.spmm(dev(A.rowptr), dev(A.colidx), dev(vals), Bp[:, :64], out=Cp[:, :64], variant="rowgroup")
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B[:, :64])
    assert np.array_equal(Cp[:, :64].cpu().numpy().astype(np.float64), want)
    assert torch.all(Cp[:, 64:] == 7.0)
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    gb.spmm(z, z[:0], torch.zeros(0, device="cuda"), Bp, variant="rowgroup")  # no rows: nothing launched


def test_rowgroup_rejected_for_sddmm(gb):
    A = gen.csr_uniform(64, 64, 0.9, seed=611)
    X = dev(gen.dense_normal(64, 32, 612))
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        gb.sddmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), X, X, variant="rowgroup")


CHOICES = {
    "uniform_41_per_row": (lambda: gen.csr_uniform(4096, 4096, 0.99, seed=621), "rowsplit"),
    "powerlaw": (lambda: gen.csr_powerlaw(8192, 8192, 0.99, seed=622), "merge"),
    "hypersparse": (lambda: gen.csr_uniform(65536, 65536, 0.99999, seed=623), "rowgroup"),
    "short_with_one_long_row": (lambda: gen.csr_from_lengths(np.r_[np.full(5000, 3), [3000]], 4000, seed=624),
                                "merge"),
}


@pytest.mark.parametrize("name", list(CHOICES))
def test_auto_choice_statistics_and_result(gb, name):
    make, expected = CHOICES[name]
    A = make()
    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    gb.auto_forget()
    choice, st = gb.auto_choice(rp, A.K, ci)
    lens = np.diff(A.rowptr.astype(np.int64))
    assert st == {"rows": A.M, "nnz": A.nnz, "sum_sq_lengths": int((lens * lens).sum()),
                  "max_length": int(lens.max()), "empty_rows": int((lens == 0).sum())}
    assert choice == expected
    B = gen.dense_normal(A.K, 64, 625)
    C = gb.spmm(rp, ci, v, dev(B)).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL32, f"auto on {name}")
    # the kept choice is what the next call uses, and gives the same bits as naming it
    C2 = gb.spmm(rp, ci, v, dev(B), variant=expected).cpu().numpy()
    assert np.array_equal(C, C2)


def test_auto_under_capture_does_not_synchronise(gb):
    """An unmeasured pattern inside a CUDA-graph capture takes the row split without
    synchronising; replays give the oracle's result."""
    import torch

    A = gen.csr_powerlaw(3000, 3000, 0.99, seed=626)
    vals = gen.vals_int(A.nnz, 627)
    B = gen.dense_int(A.K, 64, 628)
    rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(vals), dev(B)
    C = torch.empty((A.M, 64), device="cuda")
    gb.auto_forget()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            gb.spmm(rp, ci, v, Bd, out=C)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), want)
    assert gb.auto_choice(rp, A.K, ci)[0] == "merge"  # measured now, outside the capture


def test_tc_plan_residual_auto_measured_at_creation(gb):
    """A BF16 plan measures its residual's split when it is created, so its executions can
    be captured into a CUDA graph straight away."""
    import torch

    A = gen.csr_clustered(1024, 1024, 0.9, seed=629)
    vals = gen.vals_int(A.nnz, 630)
    B = gen.dense_int(A.K, 128, 631)
    bf = lambda a: dev(oracle.bf16_round(a).view(np.int16)).view(torch.bfloat16)
    gb.auto_forget()
    plan = gb.TcPlan(dev(A.rowptr), dev(A.colidx), bf(vals), A.K)
    Bd = bf(B)
    C = torch.empty((A.M, 128), device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            plan.execute(Bd, out=C, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), want)


SDDMM_CHOICES = {
    "uniform_41_per_row": (lambda: gen.csr_uniform(4096, 4096, 0.99, seed=641), "rowsplit"),
    "powerlaw": (lambda: gen.csr_powerlaw(8192, 8192, 0.99, seed=642), "merge"),
    "short_rows": (lambda: gen.csr_uniform(20000, 20000, 0.999, seed=643), "entry"),
}


@pytest.mark.parametrize("name", list(SDDMM_CHOICES))
def test_auto_sddmm_choice_and_result(gb, name):
    make, expected = SDDMM_CHOICES[name]
    A = make()
    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    gb.auto_forget()
    assert gb.auto_choice(rp, A.K, ci, op="sddmm")[0] == expected
    X, Y = gen.dense_normal(A.M, 64, 644), gen.dense_normal(A.K, 64, 645)
    out = gb.sddmm(rp, ci, v, dev(X), dev(Y)).cpu().numpy()
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, X, Y)
    assert_within(out, ref, sc, TOL32, f"auto sddmm on {name}")
    out2 = gb.sddmm(rp, ci, v, dev(X), dev(Y), variant=expected).cpu().numpy()
    assert np.array_equal(out, out2)


def test_auto_follows_a_new_pattern_at_the_same_addresses(gb):
    """A caller that writes another pattern into the same arrays (as a caching allocator
    does when it hands a freed block of the same size to a new matrix) gets a correct result
    on every call, and the new pattern's own choice once the re-measurement queued by an
    earlier call has arrived."""
    import torch

    U = gen.csr_uniform(8192, 8192, 0.99, seed=651)
    P = gen.csr_powerlaw(8192, 8192, 0.99, seed=652)
    assert U.nnz == P.nnz
    B = gen.dense_normal(8192, 64, 653)
    rp, ci, v, Bd = dev(U.rowptr), dev(U.colidx), dev(U.vals), dev(B)
    gb.auto_forget()
    assert gb.auto_choice(rp, 8192, ci)[0] == "rowsplit"
    gb.spmm(rp, ci, v, Bd)  # queues a re-measurement of the uniform pattern
    torch.cuda.synchronize()
    rp.copy_(dev(P.rowptr))
    ci.copy_(dev(P.colidx))
    v.copy_(dev(P.vals))
    ref, sc = oracle.spmm(P.rowptr, P.colidx, P.vals, B)
    choices = []
    for _ in range(3):
        C = gb.spmm(rp, ci, v, Bd).cpu().numpy()  # each result is right whatever the split
        assert_within(C, ref, sc, TOL32, "auto after the pattern changed")
        torch.cuda.synchronize()
        choices.append(gb.auto_choice(rp, 8192, ci)[0])
    assert choices[-1] == "merge", choices


def test_auto_rule_for_a_b_past_l2(gb):
    """Even rows gathered from a B of more than 192 MB in rows of 256 bytes or more take the
    row groups, 128-byte rows from a B past 96 MB the merge path; a B that fits L2 keeps the
    row split."""
    A = gen.csr_uniform(4096, 4096, 0.99, seed=661)
    rp, ci = dev(A.rowptr), dev(A.colidx)
    gb.auto_forget()
    assert gb.auto_choice(rp, A.K, ci, b_bytes=512 << 20, row_bytes=512)[0] == "rowgroup"
    assert gb.auto_choice(rp, A.K, ci, b_bytes=512 << 20, row_bytes=128)[0] == "merge"
    assert gb.auto_choice(rp, A.K, ci, b_bytes=64 << 20, row_bytes=128)[0] == "rowsplit"
    assert gb.auto_choice(rp, A.K, ci, b_bytes=64 << 20, row_bytes=512)[0] == "rowsplit"
    P = gen.csr_powerlaw(4096, 4096, 0.99, seed=662)
    assert gb.auto_choice(dev(P.rowptr), P.K, dev(P.colidx), b_bytes=512 << 20, row_bytes=512)[0] == "merge"


def test_auto_sddmm_keeps_the_row_split_for_a_y_past_l2(gb):
    A = gen.csr_uniform(4096, 4096, 0.99, seed=663)
    rp, ci = dev(A.rowptr), dev(A.colidx)
    gb.auto_forget()
    for yb, rb in ((512 << 20, 512), (512 << 20, 128), (64 << 20, 512)):
        assert gb.auto_choice(rp, A.K, ci, op="sddmm", b_bytes=yb, row_bytes=rb)[0] == "rowsplit"

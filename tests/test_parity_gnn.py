"""GPU parity of the batched graph chain (one persistent launch replayed from a CUDA graph).

Per graph: E = S o (H H^T) on the pattern of S (Eq. 2 with X = Y = H), then O = E H
(Eq. 1 with the values E); H and O in BF16, E and accumulation in FP32.  E is held to the
FP32 tolerance (1e-5 of sum |s||h_i||h_j|).  O is held to the BF16 tolerance (1e-2) of a
scale that also carries E's own error, sum_j (|E_ij| + scale(E_ij)) |H_j|, and to its
rounding: |O - O_ref| <= 2^-8 |O_ref| + 1e-5 * that scale.

The GAT-style form (softmax of each row's scores between the products) is held per row:
a weight's relative error is at most twice the scores' error (1e-5 of the row's largest
score scale, once for the entry and once through the normaliser) plus the FP32 rounding of
exp2, the row's sum (deg terms) and the division; O's error is that times sum_j alpha_ij
|H_j|, plus FP32 accumulation and BF16 rounding.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def _bf16(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)


def build_batch(graphs, seed, integer=False):
    """Host inputs and device tensors for a list of (CSR, width)."""
    import torch

    rng = np.random.default_rng(seed)
    host, devs = [], []
    for k, (A, N) in enumerate(graphs):
        if integer:
            H = rng.integers(-2, 3, size=(A.M, N)).astype(np.float32)
            sv = rng.integers(1, 4, size=A.nnz).astype(np.float32)
        else:
            H = gen.dense_normal(A.M, N, seed * 1000 + k)
            sv = A.vals
        Hb = _bf16(H)
        host.append((A, sv, Hb.float().numpy().astype(np.float64)))
        devs.append((dev(A.rowptr), dev(A.colidx), dev(sv), Hb.cuda(),
                     torch.empty((A.M, N), dtype=torch.bfloat16, device="cuda"),
                     torch.empty(A.nnz, dtype=torch.float32, device="cuda")))
    return host, devs


def check_graph(A, sv, Hd, E_gpu, O_gpu, exact=False):
    E_ref, sE = oracle.sddmm(A.rowptr, A.colidx, sv, Hd, Hd)
    O_ref, _ = oracle.spmm(A.rowptr, A.colidx, E_ref, Hd)
    if exact:
        assert np.array_equal(E_gpu.astype(np.float64), E_ref)
        want = _bf16(O_ref.astype(np.float32)).float().numpy()
        assert np.array_equal(O_gpu, want)
        return
    z = sE == 0
    assert np.all(E_gpu[z] == 0)
    assert np.all(np.abs(E_gpu - E_ref)[~z] <= 1e-5 * sE[~z])
    scale, _ = oracle.spmm(A.rowptr, A.colidx, np.abs(E_ref) + sE, np.abs(Hd))
    err = np.abs(O_gpu.astype(np.float64) - O_ref)
    assert np.all(err <= 1e-2 * scale + 1e-30)
    assert np.all(err <= 2.0**-8 * np.abs(O_ref) + 1e-5 * scale + 1e-30)


def small_graphs(seed, G=10, widths=(64, 128, 256, 72, 200)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(G):
        n = int(rng.integers(100, 3000))
        out.append((gen.gnn_graph(n, seed * 100 + k), int(widths[k % len(widths)])))
    return out


def test_gnn_chain_random(gb):
    graphs = small_graphs(501)
    host, devs = build_batch(graphs, 502)
    plan = gb.GnnPlan(devs)
    info = plan.info()
    assert info["graphs"] == len(graphs) and info["edges"] == sum(A.nnz for A, _ in graphs)
    plan.execute()
    import torch

    torch.cuda.synchronize()
    for (A, sv, Hd), d in zip(host, devs):
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy())


def test_gnn_chain_integers_bit_exact(gb):
    graphs = small_graphs(503, G=6)
    host, devs = build_batch(graphs, 504, integer=True)
    gb.gnn_sddmm_spmm_batched(devs)
    for (A, sv, Hd), d in zip(host, devs):
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy(), exact=True)


@pytest.mark.parametrize("N", [64, 128, 256])
def test_gnn_chain_row_lengths_bit_exact(gb, N):
    """Empty rows and rows of 1 to 5, 31 to 33 and 70 edges in every position of a tile: the
    short rows (at most as many edges as a group step takes) go G to a warp pass, the others
    one after another, and both give the oracle's integers exactly."""
    rng = np.random.default_rng(508)
    lengths = rng.choice(np.array([0, 1, 1, 1, 2, 2, 3, 4, 5, 31, 32, 33, 70]), size=700)
    A = gen.csr_from_lengths(lengths, 700, seed=509)
    host, devs = build_batch([(A, N)], 510, integer=True)
    for ept in (0, 40):
        plan = gb.GnnPlan(devs, edges_per_tile=ept) if ept else gb.GnnPlan(devs)
        plan.execute()
        import torch

        torch.cuda.synchronize()
        (A, sv, Hd), d = host[0], devs[0]
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy(), exact=True)


@pytest.mark.parametrize("edges_per_tile", [1, 64, 100000])
def test_gnn_replay_and_tiles(gb, edges_per_tile):
    """Replays of the recorded graph follow new data in the same buffers; any tile size."""
    import torch

    graphs = small_graphs(505, G=5)
    host, devs = build_batch(graphs, 506, integer=True)
    plan = gb.GnnPlan(devs, edges_per_tile=edges_per_tile)
    plan.execute()
    plan.execute()
    torch.cuda.synchronize()
    for (A, sv, Hd), d in zip(host, devs):
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy(), exact=True)
    # new features in the same buffers
    rng = np.random.default_rng(507)
    for i, (A, sv, Hd) in enumerate(host):
        H2 = rng.integers(-2, 3, size=Hd.shape).astype(np.float32)
        devs[i][3].copy_(_bf16(H2).cuda())
        host[i] = (A, sv, H2.astype(np.float64))
    plan.execute()
    torch.cuda.synchronize()
    for (A, sv, Hd), d in zip(host, devs):
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy(), exact=True)


def test_gnn_batch_configuration_sampled(gb):
    """The batch configuration: 512 graphs, 1,000..50,000 nodes (log-uniform), power-law
    degrees (mean 16, max 2,048), widths 64/128/256; 12 graphs checked against the oracle."""
    import torch

    graphs = gen.gnn_batch(G=512, seed=3000)
    host, devs = build_batch(graphs, 3001)
    plan = gb.GnnPlan(devs)
    plan.execute()
    torch.cuda.synchronize()
    pick = np.random.default_rng(3002).choice(len(graphs), 12, replace=False)
    for i in pick:
        A, sv, Hd = host[i]
        d = devs[i]
        check_graph(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy())


# ---- GAT-style chain: softmax of each row's scores between SDDMM and SpMM ----------------------

def check_gat(A, sv, Hd, E_gpu, O_gpu):
    """alpha (E_gpu) against the oracle's row softmax of the FP64 scores, relative to a row
    tolerance that carries the scores' FP32 error (1e-5 of their scale, twice: the entry and
    the row's normaliser); O against alpha H with that error and BF16 rounding."""
    alpha, O_ref, sO = oracle.gat_chain(A.rowptr, A.colidx, sv, Hd)
    _, sE = oracle.sddmm(A.rowptr, A.colidx, sv, Hd, Hd)
    lens = A.row_lengths()
    row_scale = np.zeros(A.M)
    nz = lens > 0
    row_scale[nz] = np.maximum.reduceat(sE, A.rowptr[:-1][nz])
    tol_row = 2e-5 * row_scale + 1e-6 + lens * 2.0**-24
    tol_e = np.repeat(tol_row, lens)
    assert np.all(np.abs(E_gpu - alpha) <= tol_e * alpha + 1e-7)
    err = np.abs(O_gpu.astype(np.float64) - O_ref)
    assert np.all(err <= 2.0**-8 * np.abs(O_ref) + (tol_row[:, None] + 1e-5) * sO + 1e-30)
    assert np.all(O_gpu[~nz] == 0)


@pytest.mark.parametrize("one_shot", [False, True])
def test_gat_chain_random(gb, one_shot):
    graphs = small_graphs(511)
    host, devs = build_batch(graphs, 512)
    if one_shot:
        gb.gnn_gat_batched(devs)
    else:
        plan = gb.GnnPlan(devs, softmax=True)
        plan.execute()
        plan.execute()  # replay: E is overwritten with the same weights
    import torch

    torch.cuda.synchronize()
    for (A, sv, Hd), d in zip(host, devs):
        check_gat(A, sv, Hd, d[5].cpu().numpy(), d[4].float().cpu().numpy())


def test_gat_chain_rows_and_special_cases(gb):
    """Empty rows, single-edge rows (weight exactly 1), rows longer than a 32-edge chunk,
    all-zero scores (weights 1/deg), and every width layout."""
    import torch

    rng = np.random.default_rng(513)
    graphs = []
    for k, N in enumerate((64, 128, 256, 8)):
        n = 400
        lengths = rng.integers(0, 6, n)
        lengths[:40] = 0
        lengths[40:80] = 1
        lengths[80:90] = rng.integers(33, 120, 10)
        graphs.append((gen.csr_from_lengths(lengths, n, seed=514 + k), N))
    host, devs = build_batch(graphs, 515)
    # one graph with zero values: every score 0, weights 1 / deg
    A0, N0 = graphs[0]
    devs[0] = (devs[0][0], devs[0][1], torch.zeros(A0.nnz, device="cuda"), *devs[0][3:])
    host[0] = (A0, np.zeros(A0.nnz, np.float32), host[0][2])
    gb.gnn_gat_batched(devs)
    torch.cuda.synchronize()
    for (A, sv, Hd), d in zip(host, devs):
        E = d[5].cpu().numpy()
        check_gat(A, sv, Hd, E, d[4].float().cpu().numpy())
        single = np.repeat(A.row_lengths() == 1, A.row_lengths())
        assert np.all(E[single] == 1.0)
    lens0 = host[0][0].row_lengths()
    want = np.repeat(np.where(lens0 > 0, 1.0 / np.maximum(lens0, 1), 0), lens0).astype(np.float32)
    assert np.array_equal(devs[0][5].cpu().numpy(), want)


def test_gat_plan_rejects_unknown_flags(gb):
    import ctypes

    from paper_2604_27985_gb300._lib import lib

    h = ctypes.c_void_p()
    assert lib.gbsp_gnn_plan_create_ex(0, None, None, None, None, 0, 2, None, ctypes.byref(h)) == -1

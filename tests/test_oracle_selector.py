"""Pins for the selector oracle: a hand-computed feature example, feature invariants, the
MLP gradient against finite differences and torch autograd, Adam against torch.optim."""
import os

import numpy as np
import pytest

import gen
from oracle import selector as osel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_features_worked_example():
    d = {}
    for line in open(os.path.join(GOLDEN, "features_4x16.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = [float(t) for t in v]
    f = osel.features(np.array(d["rowptr"], np.int32), np.array(d["colidx"], np.int32), 4, 16, 64, 1)
    want = [d["f0"][0], d["f1"][0], np.log2(d["f2_log2_of"][0]), np.log2(d["f3_log2_of"][0]),
            np.log2(d["f4_log2_of"][0]), np.log2(1 + np.sqrt(d["f5_log2_of_1_plus_sqrt"][0])),
            np.sqrt(d["f6_sqrt_over"][0]) / d["f6_sqrt_over"][1], d["f7"][0], d["f8"][0], d["f9"][0],
            d["f10"][0], d["f11"][0], d["f12_ratio"][0] / d["f12_ratio"][1], d["f13_ratio"][0] / d["f13_ratio"][1],
            d["f14"][0], d["f15"][0]]
    np.testing.assert_allclose(f, want, rtol=1e-14, atol=0)


def test_features_invariants():
    n = 500
    diag = osel.features(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), n, n, 32)
    assert diag[6] == 0 and diag[10] == 0 and diag[11] == 0 and diag[12] == 0 and diag[13] == 0 and diag[9] == 0
    # a full band of width 3 (i-1, i, i+1): every consecutive pair is 1 apart, and each entry
    # but the last row's and the ones past the band edge has a vertical neighbour
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
    A = gen.csr_from_triplets(n, n, rows, cols, np.ones(len(rows)))
    f = osel.features(A.rowptr, A.colidx, n, n, 32)
    assert f[12] == 1.0
    brute = sum(1 for i, j in zip(rows, cols) if i + 1 < n and abs(j - (i + 1)) <= 1)
    assert f[13] == brute / len(rows)
    U = gen.csr_uniform(1000, 800, 0.9, seed=1)
    assert osel.features(U.rowptr, U.colidx, 1000, 800, 16)[6] < 0.01


def _data(seed, n=40):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(osel.N_PARAMS) * 0.2
    x = rng.standard_normal((n, osel.F))
    t = rng.standard_normal((n, osel.V))
    m = (rng.random((n, osel.V)) > 0.2).astype(np.float64)
    return w, x, t, m


def test_gradient_matches_finite_differences():
    w, x, t, m = _data(1)
    g = osel.gradient(w, x, t, m)
    rng = np.random.default_rng(2)
    for k in rng.choice(osel.N_PARAMS, 60, replace=False):
        e = np.zeros_like(w)
        e[k] = 1e-6
        fd = (osel.loss(w + e, x, t, m) - osel.loss(w - e, x, t, m)) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def _torch_mlp(torch, w):
    p = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in osel.unpack(w).items()}
    return p


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    w, x, t, m = _data(3)
    p = _torch_mlp(torch, w)
    X, T, Mk = (torch.tensor(a) for a in (x, t, m))
    h1 = torch.relu(X @ p["W1"].T + p["b1"])
    h2 = torch.relu(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["W3"].T + p["b3"]
    loss = (Mk * (y - T) ** 2).sum() / Mk.sum()
    loss.backward()
    g_t = np.concatenate([p[k].grad.numpy().ravel() for k, _ in osel.SIZES])
    np.testing.assert_allclose(osel.gradient(w, x, t, m), g_t, rtol=1e-10, atol=1e-12)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    w, x, t, m = _data(4, n=50)
    norm = np.concatenate([np.zeros(osel.F), np.ones(osel.F)])
    order = np.random.default_rng(5).permutation(50)
    steps, batch, lr = 6, 16, 1e-2
    w_o, _ = osel.train(w, np.zeros(2 * osel.N_PARAMS), norm, x, t, m, order, steps, batch, lr)
    p = _torch_mlp(torch, w)
    params = [p[k] for k, _ in osel.SIZES]
    opt = torch.optim.Adam(params, lr=lr, betas=(0.9, 0.999), eps=1e-8)
    for step in range(steps):
        base = (step * batch) % 50
        idx = order[(base + np.arange(batch)) % 50]
        X, T, Mk = (torch.tensor(a[idx]) for a in (x, t, m))
        opt.zero_grad()
        h1 = torch.relu(X @ p["W1"].T + p["b1"])
        h2 = torch.relu(h1 @ p["W2"].T + p["b2"])
        y = h2 @ p["W3"].T + p["b3"]
        ((Mk * (y - T) ** 2).sum() / Mk.sum()).backward()
        opt.step()
    w_t = np.concatenate([q.detach().numpy().ravel() for q in params])
    np.testing.assert_allclose(w_o, w_t, rtol=1e-9, atol=1e-12)

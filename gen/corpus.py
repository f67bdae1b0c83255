"""Seeded corpus of matrices for training and judging the kernel selector.

Each corpus entry draws (from numpy, seeded by (seed, index)): rows n log-uniform in
[4,096, 262,144] (square), sparsity in {90, 99, 99.9}%, a structure in {uniform, power-law,
banded, block}, a dense width N in {32, 64, 128, 256, 512} and a value type in {FP32, BF16}.
Draws whose nonzero count passes `max_nnz` (default 2^24) or whose nnz * N passes
`max_work` (default 2^31) are redrawn, which bounds the time the autotuner spends per
matrix; the number of redraws is reported.  The column indices are drawn on the device with
torch (uniform per row, or inside a band, or as dense b x b blocks) and sorted within rows;
repeated columns are allowed (they are separate terms of the product).  Nothing here
computes any part of SpMM.
"""
from __future__ import annotations

import math

import numpy as np

from .csr import _largest_remainder, nnz_for, powerlaw_lengths

STRUCTURES = ("uniform", "powerlaw", "banded", "block")
WIDTHS = (32, 64, 128, 256, 512)
SPARSITIES = (0.9, 0.99, 0.999)


def corpus_spec(index: int, seed: int, max_nnz: int = 1 << 24, max_work: int = 1 << 31) -> dict:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(index), 7])))
    redraws = 0
    while True:
        n = int(round(math.exp(rng.uniform(math.log(4096), math.log(262144)))))
        sp = float(rng.choice(SPARSITIES))
        st = str(rng.choice(STRUCTURES))
        N = int(rng.choice(WIDTHS))
        dt = int(rng.integers(0, 2))
        T = nnz_for(n, n, sp)
        if T <= max_nnz and T * N <= max_work:
            break
        redraws += 1
    return {"index": index, "seed": seed, "n": n, "sparsity": sp, "structure": st, "N": N, "dtype": dt,
            "nnz_target": T, "redraws": redraws}


def extrapolation_spec(index: int, seed: int) -> dict:
    """A held-out matrix outside the corpus's range of rows: 1,048,576 x 1,048,576 at 99.99%,
    99.999% or 99.9999% sparsity, one of the four structures, N in {32, 64, 128}, FP32 or
    BF16 (drawn from (seed, index) as corpus_spec draws)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(index), 13])))
    n = 1 << 20
    sp = float(rng.choice((0.9999, 0.99999, 0.999999)))
    st = str(rng.choice(STRUCTURES))
    N = int(rng.choice((32, 64, 128)))
    dt = int(rng.integers(0, 2))
    return {"index": index, "seed": seed, "n": n, "sparsity": sp, "structure": st, "N": N, "dtype": dt,
            "nnz_target": nnz_for(n, n, sp), "redraws": 0}


def corpus_matrix(spec: dict, device="cuda"):
    """(rowptr, colidx, vals) torch tensors on the device for one corpus entry."""
    import torch

    n, T, st = spec["n"], spec["nnz_target"], spec["structure"]
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec["seed"], spec["index"], 11])))
    g = torch.Generator(device=device)
    g.manual_seed(int(rng.integers(0, 2**62)))
    if st == "block":
        b = int(rng.choice([8, 16, 32]))
        nb_side = n // b
        nblk = max(1, min(nb_side * nb_side, int(round(T / (b * b)))))
        ids = np.sort(rng.choice(nb_side * nb_side, nblk, replace=False)).astype(np.int64)
        br, bc = ids // nb_side, ids % nb_side
        ii, jj = np.divmod(np.arange(b * b, dtype=np.int64), b)
        rows = torch.from_numpy((br[:, None] * b + ii[None, :]).ravel()).to(device)
        cols = torch.from_numpy((bc[:, None] * b + jj[None, :]).ravel()).to(device)
    else:
        if st == "uniform":
            base, extra = divmod(T, n)
            lengths = np.full(n, base, dtype=np.int64)
            lengths[rng.permutation(n)[:extra]] += 1
        elif st == "powerlaw":
            lengths, _, _ = powerlaw_lengths(rng, n, n, T)
        else:  # banded: bandwidth 1-5% of n, entries uniform inside the band
            bw = max(1, int(round(rng.uniform(0.01, 0.05) * n)))
            centre = np.arange(n, dtype=np.int64)
            lo = np.maximum(centre - bw, 0)
            width = np.minimum(centre + bw + 1, n) - lo
            T = min(T, int(width.sum()))
            lengths = _largest_remainder(width * (T / width.sum()), T)
            lengths = np.minimum(lengths, width)
        rows = torch.repeat_interleave(torch.arange(n, device=device), torch.from_numpy(lengths).to(device))
        u = torch.rand(rows.shape[0], generator=g, device=device, dtype=torch.float64)
        if st == "banded":
            lo_t = torch.from_numpy(lo).to(device)[rows]
            w_t = torch.from_numpy(width).to(device)[rows]
            cols = lo_t + torch.minimum((u * w_t).long(), w_t - 1)
        else:
            cols = torch.minimum((u * n).long(), torch.tensor(n - 1, device=device))
    keys = torch.sort(rows * n + cols).values
    rows, cols = keys // n, keys % n
    counts = torch.bincount(rows, minlength=n)
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(counts, 0)
    vals = torch.rand(cols.shape[0], generator=g, device=device) * 2 - 1
    return rowptr.to(torch.int32), cols.to(torch.int32), vals.to(torch.float32)

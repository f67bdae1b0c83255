"""Seeded CSR patterns and dense fills with the shapes of the paper's workloads.

The paper measures on random sparse matrices and random dense operands (Section V-A:
random N x N sparse matrices, K = N, D = 256).  Everything here is drawn from numpy's
PCG64 through ``SeedSequence([seed, stream])`` so that the same seed gives the same
matrix on every host (x86_64 and aarch64 alike).

Readings of what the paper leaves open (each one is listed in the design notes):

* nnz of an ``s``-sparse M x K matrix is ``round((1 - s) * M * K)``.
* "uniform" rows: every row gets ``T // M`` entries, and ``T % M`` rows chosen by a seeded
  permutation get one more; columns are uniform without replacement and sorted.
* "power-law" rows: lengths drawn from P(l) ~ l^-alpha on [1, cap], rescaled to hit T
  exactly (largest remainder), clipped at min(cap, K) with the excess handed to the
  unclipped rows; when T cannot fit under the cap the cap is raised to K.
* "clustered": aligned 16 x 8 blocks holding 51 of their 128 slots, half of T inside
  blocks, the rest uniform over positions outside the chosen blocks.
* GNN graphs: node counts log-uniform, degrees P(d) ~ d^-alpha on [1, min(2048, n-1)]
  with alpha fixed so the mean on [1, 2048] is 16, no self loops, row-normalised values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Streams of one seed: each kind of draw has its own so that adding a draw of one kind
# does not shift the others.
_S_LENGTHS, _S_COLS, _S_VALS, _S_BLOCKS, _S_DENSE, _S_GRAPH = range(6)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


@dataclass
class CSR:
    """A sparse matrix in CSR form: int32 row pointers and column indices, FP32 values."""

    M: int
    K: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    def csr_bytes(self, value_bytes: int = 4) -> int:
        """Bytes of the CSR arrays: (index + value) per nonzero plus M+1 row pointers."""
        return (4 + value_bytes) * self.nnz + 4 * (self.M + 1)

    def with_vals(self, vals: np.ndarray) -> "CSR":
        return CSR(self.M, self.K, self.rowptr, self.colidx, np.ascontiguousarray(vals), dict(self.meta))


def nnz_for(M: int, K: int, sparsity: float | None = None, density: float | None = None) -> int:
    """Number of stored entries of an M x K matrix at the given sparsity (or density)."""
    if density is None:
        if sparsity is None:
            raise ValueError("give sparsity or density")
        density = 1.0 - sparsity
    return int(round(density * M * K))


def _largest_remainder(x: np.ndarray, total: int) -> np.ndarray:
    """Integers summing to ``total`` that round the non-negative reals ``x``."""
    f = np.floor(x).astype(np.int64)
    r = int(total - f.sum())
    if r > 0:
        order = np.argsort(-(x - f), kind="stable")
        f[order[:r]] += 1
    elif r < 0:
        order = np.argsort(x - f, kind="stable")
        order = order[f[order] > 0]
        f[order[:-r]] -= 1
    return f


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + neighbour compare; much faster than np.unique here)."""
    s = np.sort(keys)
    if s.shape[0] == 0:
        return s
    keep = np.empty(s.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _uniform_lengths(rng: np.random.Generator, M: int, T: int) -> np.ndarray:
    base, extra = divmod(T, M)
    lengths = np.full(M, base, dtype=np.int64)
    if extra:
        lengths[rng.permutation(M)[:extra]] += 1
    return lengths


def _sample_columns(rng, lengths, K, lo=None, width=None, exclude_self=False, forbidden=None):
    """Sorted, distinct column indices per row.

    Row r draws ``lengths[r]`` columns uniformly from ``[lo[r], lo[r] + width[r])`` (the
    whole ``[0, K)`` by default), skipping column r itself when ``exclude_self`` is set and
    any (row, col) for which ``forbidden(rows, cols)`` is true.  Sparse rows are drawn
    together with rejection of repeats; rows that take more than half of their range are
    drawn one at a time.
    """
    M = lengths.shape[0]
    lengths = lengths.astype(np.int64)
    if lo is None:
        lo = np.zeros(M, dtype=np.int64)
        width = np.full(M, K, dtype=np.int64)
    avail = width - (1 if exclude_self else 0)
    if np.any(lengths > avail) and forbidden is None:
        raise ValueError("a row asks for more columns than it has")
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(lengths, out=rowptr[1:])
    T = int(rowptr[-1])
    colidx = np.empty(T, dtype=np.int64)
    dense = (lengths * 2 > avail) & (lengths > 0)
    sparse_rows = np.nonzero(~dense & (lengths > 0))[0]

    def draw(rows):
        r64 = rows.astype(np.int64)
        u = rng.random(rows.shape[0])
        c = lo[r64] + np.minimum((u * avail[r64]).astype(np.int64), avail[r64] - 1)
        if exclude_self:
            c = c + (c >= r64)
        if forbidden is not None:
            keep = ~forbidden(r64, c)
            r64, c = r64[keep], c[keep]
        return r64 * K + c

    if sparse_rows.size:
        target = np.zeros(M, dtype=np.int64)
        target[sparse_rows] = lengths[sparse_rows]
        keys = draw(np.repeat(np.arange(M, dtype=np.int64), target))
        while True:
            keys = _sorted_unique(keys)
            counts = np.bincount(keys // K, minlength=M)
            deficit = target - counts
            short = int(deficit.sum())
            if short == 0:
                break
            keys = np.concatenate([keys, draw(np.repeat(np.arange(M, dtype=np.int64), deficit))])
        mask = np.repeat(~dense, lengths)
        colidx[mask] = keys % K
    for r in np.nonzero(dense)[0]:
        L = int(lengths[r])
        cand = np.arange(lo[r], lo[r] + width[r], dtype=np.int64)
        if exclude_self:
            cand = cand[cand != r]
        if forbidden is not None:
            cand = cand[~forbidden(np.full(cand.shape[0], r, dtype=np.int64), cand)]
        pick = np.sort(rng.choice(cand.shape[0], L, replace=False))
        colidx[rowptr[r]:rowptr[r + 1]] = cand[pick]
    return rowptr, colidx


def _finish(M, K, rowptr64, colidx64, vals, meta) -> CSR:
    if rowptr64[-1] >= 2**31:
        raise ValueError("nnz exceeds the int32 row-pointer range")
    return CSR(M, K, rowptr64.astype(np.int32), colidx64.astype(np.int32),
               np.ascontiguousarray(vals, dtype=np.float32), meta)


def _uniform_vals(seed: int, n: int) -> np.ndarray:
    """Values uniform on [-1, 1) in FP32."""
    rng = _rng(seed, _S_VALS)
    return (rng.random(n, dtype=np.float32) * np.float32(2.0) - np.float32(1.0)).astype(np.float32)


def csr_from_lengths(lengths, K: int, seed: int, **kw) -> CSR:
    """CSR with the given row lengths, uniform columns and U[-1, 1] values."""
    lengths = np.asarray(lengths, dtype=np.int64)
    rowptr, colidx = _sample_columns(_rng(seed, _S_COLS), lengths, K, **kw)
    return _finish(lengths.shape[0], K, rowptr, colidx, _uniform_vals(seed, int(rowptr[-1])),
                   {"kind": "lengths", "seed": seed})


def csr_uniform(M: int, K: int, sparsity: float | None = None, seed: int = 0,
                density: float | None = None, nnz: int | None = None) -> CSR:
    """Uniform rows: T // M entries per row, T % M rows one longer, columns uniform."""
    T = nnz if nnz is not None else nnz_for(M, K, sparsity, density)
    lengths = _uniform_lengths(_rng(seed, _S_LENGTHS), M, T)
    rowptr, colidx = _sample_columns(_rng(seed, _S_COLS), lengths, K)
    return _finish(M, K, rowptr, colidx, _uniform_vals(seed, T),
                   {"kind": "uniform", "seed": seed, "sparsity": sparsity})


def _powerlaw_draw(rng, n: int, alpha: float, lo: int, hi: int) -> np.ndarray:
    ells = np.arange(lo, hi + 1, dtype=np.float64)
    cdf = np.cumsum(ells ** (-alpha))
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, rng.random(n), side="right")
    return ells[np.minimum(idx, ells.shape[0] - 1)].astype(np.int64)


def powerlaw_lengths(rng, M: int, K: int, T: int, alpha: float = 1.5, cap: int = 4096):
    """Row lengths with a truncated power-law shape summing to exactly T."""
    lmax = min(cap, K)
    raised = False
    if T > M * lmax:
        lmax, raised = K, True
    if T > M * K:
        raise ValueError("T does not fit in an M x K matrix")
    draws = _powerlaw_draw(rng, M, alpha, 1, cap).astype(np.float64)
    lengths = _largest_remainder(draws * (T / draws.sum()), T)
    for _ in range(10000):
        over = lengths > lmax
        if not over.any():
            break
        excess = int((lengths[over] - lmax).sum())
        lengths[over] = lmax
        free = lengths < lmax
        w = lengths[free].astype(np.float64)
        if w.sum() == 0:
            w = np.ones_like(w)
        lengths[free] += _largest_remainder(w * (excess / w.sum()), excess)
    assert int(lengths.sum()) == T and int(lengths.max()) <= lmax
    return lengths, lmax, raised


def csr_powerlaw(M: int, K: int, sparsity: float, seed: int = 0, alpha: float = 1.5,
                 cap: int = 4096) -> CSR:
    """Power-law rows (Zipf exponent ``alpha``, capped), columns uniform per row."""
    T = nnz_for(M, K, sparsity)
    lengths, lmax, raised = powerlaw_lengths(_rng(seed, _S_LENGTHS), M, K, T, alpha, cap)
    rowptr, colidx = _sample_columns(_rng(seed, _S_COLS), lengths, K)
    return _finish(M, K, rowptr, colidx, _uniform_vals(seed, T),
                   {"kind": "powerlaw", "seed": seed, "sparsity": sparsity, "alpha": alpha,
                    "cap": int(lmax), "cap_raised": bool(raised)})


def csr_clustered(M: int, K: int, sparsity: float, seed: int = 0, bh: int = 16, bw: int = 8,
                  fill: int = 51, block_share: float = 0.5) -> CSR:
    """Aligned bh x bw blocks with ``fill`` random slots each, holding ``block_share`` of
    the nonzeros; the rest uniform over the positions outside the chosen blocks."""
    if M % bh or K % bw:
        raise ValueError("block grid must tile the matrix")
    T = nnz_for(M, K, sparsity)
    nbr, nbc = M // bh, K // bw
    nb = int(round(block_share * T / fill))
    rb = _rng(seed, _S_BLOCKS)
    chosen = np.sort(rb.choice(nbr * nbc, nb, replace=False)).astype(np.int64)
    is_block = np.zeros(nbr * nbc, dtype=bool)
    is_block[chosen] = True
    slots = np.argsort(rb.random((nb, bh * bw)), axis=1)[:, :fill].astype(np.int64)
    br, bc = chosen // nbc, chosen % nbc
    r_blk = (br[:, None] * bh + slots // bw).ravel()
    c_blk = (bc[:, None] * bw + slots % bw).ravel()
    rest = T - nb * fill
    lengths = _uniform_lengths(_rng(seed, _S_LENGTHS), M, rest)

    def forbidden(rows, cols):
        return is_block[(rows // bh) * nbc + cols // bw]

    rp_rest, ci_rest = _sample_columns(_rng(seed, _S_COLS), lengths, K, forbidden=forbidden)
    r_rest = np.repeat(np.arange(M, dtype=np.int64), lengths)
    keys = np.sort(np.concatenate([r_blk * K + c_blk, r_rest * K + ci_rest]))
    rows = keys // K
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=M), out=rowptr[1:])
    return _finish(M, K, rowptr, keys % K, _uniform_vals(seed, T),
                   {"kind": "clustered", "seed": seed, "sparsity": sparsity, "block": [bh, bw],
                    "fill": fill, "blocks": nb, "block_nnz": nb * fill})


def csr_banded(M: int, K: int, sparsity: float, seed: int = 0, band_frac: float | None = None) -> CSR:
    """Nonzeros uniform inside a band |j - i*K/M| <= b with b a fraction of n."""
    rl = _rng(seed, _S_LENGTHS)
    if band_frac is None:
        band_frac = float(rl.uniform(0.01, 0.05))
    b = max(1, int(round(band_frac * K)))
    centre = (np.arange(M, dtype=np.int64) * K) // M
    lo = np.maximum(centre - b, 0)
    hi = np.minimum(centre + b + 1, K)
    width = hi - lo
    T = min(nnz_for(M, K, sparsity), int(width.sum()))
    lengths = _uniform_lengths(rl, M, T)
    over = lengths > width
    if over.any():  # rows clipped by the matrix edge: give their excess to the others
        excess = int((lengths[over] - width[over]).sum())
        lengths[over] = width[over]
        room = width - lengths
        lengths += _largest_remainder(room * (excess / room.sum()), excess)
        lengths = np.minimum(lengths, width)
    rowptr, colidx = _sample_columns(_rng(seed, _S_COLS), lengths, K, lo=lo, width=width)
    return _finish(M, K, rowptr, colidx, _uniform_vals(seed, int(rowptr[-1])),
                   {"kind": "banded", "seed": seed, "sparsity": sparsity, "band": b})


def csr_blocked(M: int, K: int, sparsity: float, seed: int = 0, b: int | None = None) -> CSR:
    """Fully dense b x b blocks at uniform positions of the aligned block grid."""
    rb = _rng(seed, _S_BLOCKS)
    if b is None:
        b = int(rb.choice([8, 16, 32]))
    nbr, nbc = M // b, K // b
    T = nnz_for(M, K, sparsity)
    nb = min(max(1, int(round(T / (b * b)))), nbr * nbc)
    chosen = np.sort(rb.choice(nbr * nbc, nb, replace=False)).astype(np.int64)
    br, bc = chosen // nbc, chosen % nbc
    ii, jj = np.divmod(np.arange(b * b, dtype=np.int64), b)
    rows = (br[:, None] * b + ii[None, :]).ravel()
    cols = (bc[:, None] * b + jj[None, :]).ravel()
    keys = np.sort(rows * K + cols)
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(np.bincount(keys // K, minlength=M), out=rowptr[1:])
    return _finish(M, K, rowptr, keys % K, _uniform_vals(seed, keys.shape[0]),
                   {"kind": "blocked", "seed": seed, "sparsity": sparsity, "block": b})


def csr_from_triplets(M: int, K: int, rows, cols, vals, sort: bool = True) -> CSR:
    """CSR from explicit (row, col, value) entries; repeats are kept as separate entries."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float32)
    order = np.argsort(rows, kind="stable") if sort else np.arange(rows.shape[0])
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=M), out=rowptr[1:])
    return _finish(M, K, rowptr, cols[order], vals[order], {"kind": "triplets"})


def gnn_alpha(mean: float = 16.0, dmax: int = 2048) -> float:
    """Exponent of P(d) ~ d^-alpha on [1, dmax] whose mean is ``mean`` (bisection)."""
    d = np.arange(1, dmax + 1, dtype=np.float64)

    def m(a):
        w = d ** (-a)
        return float((d * w).sum() / w.sum())

    lo, hi = 1.0001, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if m(mid) > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


_ALPHA16 = None


def gnn_graph(n: int, seed: int, alpha: float | None = None, dmax_cap: int = 2048) -> CSR:
    """One graph adjacency: power-law out-degrees, uniform neighbours, no self loops,
    values 1/deg (row-normalised)."""
    global _ALPHA16
    if alpha is None:
        if _ALPHA16 is None:
            _ALPHA16 = gnn_alpha(16.0, 2048)
        alpha = _ALPHA16
    dmax = min(dmax_cap, n - 1)
    deg = _powerlaw_draw(_rng(seed, _S_LENGTHS), n, alpha, 1, dmax)
    rowptr, colidx = _sample_columns(_rng(seed, _S_COLS), deg, n, exclude_self=True)
    vals = np.repeat((1.0 / deg).astype(np.float32), deg)
    return _finish(n, n, rowptr, colidx, vals, {"kind": "gnn", "seed": seed, "alpha": alpha})


def gnn_batch(G: int = 512, seed: int = 3000, nmin: int = 1000, nmax: int = 50000,
              widths=(64, 128, 256)):
    """G graphs with log-uniform node counts and a feature width drawn per graph."""
    rg = _rng(seed, _S_GRAPH)
    ns = np.rint(np.exp(rg.uniform(math.log(nmin), math.log(nmax), size=G))).astype(np.int64)
    ws = rg.choice(np.asarray(widths, dtype=np.int64), size=G)
    return [(gnn_graph(int(ns[g]), seed * 1000 + g + 1), int(ws[g])) for g in range(G)]


def dense_normal(rows: int, cols: int, seed: int) -> np.ndarray:
    """Row-major FP32 matrix with N(0, 1) entries."""
    return _rng(seed, _S_DENSE).standard_normal((rows, cols), dtype=np.float32)


def dense_uniform(rows: int, cols: int, seed: int) -> np.ndarray:
    """Row-major FP32 matrix with U[-1, 1) entries."""
    r = _rng(seed, _S_DENSE)
    return (r.random((rows, cols), dtype=np.float32) * np.float32(2) - np.float32(1)).astype(np.float32)


def dense_int(rows: int, cols: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Row-major FP32 matrix of integers in [lo, hi] (exact in FP32, BF16 and E4M3)."""
    return _rng(seed, _S_DENSE).integers(lo, hi + 1, size=(rows, cols)).astype(np.float32)


def vals_int(n: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """FP32 integer values in [lo, hi] for the stored entries of a pattern."""
    return _rng(seed, _S_VALS).integers(lo, hi + 1, size=n).astype(np.float32)

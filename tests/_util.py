"""Helpers shared by the GPU parity tests (no SpMM / SDDMM arithmetic here)."""
import numpy as np


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_within(gpu, ref, scale, tol, what=""):
    """|gpu - ref| <= tol * scale elementwise; where scale is 0 the result must be 0.
    Returns (max, mean) of |err| / scale over the outputs with scale > 0."""
    gpu = np.asarray(gpu, dtype=np.float64)
    err = np.abs(gpu - ref)
    z = scale == 0
    assert np.all(gpu[z] == 0), f"{what}: nonzero output where the scale is 0"
    nz = ~z
    rel = err[nz] / scale[nz]
    if rel.size:
        worst = int(np.argmax(rel))
        assert rel[worst] <= tol, f"{what}: max |err|/scale {rel[worst]:.3e} > {tol:g}"
        return float(rel.max()), float(rel.mean())
    return 0.0, 0.0


def sub_csr(rowptr, colidx, vals, rows):
    """The CSR of the listed rows (for row-sampled oracle checks of large matrices)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    lens = rowptr[rows + 1] - rowptr[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    return rp.astype(np.int32), np.asarray(colidx)[idx], np.asarray(vals)[idx], idx

"""Torch-tensor front end of the C ABI: same names as the entry points, marshalling only.

Every function takes CUDA tensors, passes their device pointers and the current torch
stream (or the one given) to libgbsp.so, and returns the output tensor.  No arithmetic of
SpMM / SDDMM happens here; PyTorch only owns the memory and the stream.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import BF16, E4M3, F32, VARIANTS, Csr, Dense, Opts, check, lib

_DT = {torch.float32: F32, torch.bfloat16: BF16, torch.uint8: E4M3}
if hasattr(torch, "float8_e4m3fn"):
    _DT[torch.float8_e4m3fn] = E4M3


def _dtype(t: torch.Tensor) -> int:
    try:
        return _DT[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {t.dtype}") from None


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensors must live on a CUDA device")
    return t.data_ptr() or None


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("dense operands must be 2-D with unit column stride")
    return t.stride(0) if t.shape[0] > 1 else max(t.stride(0), t.shape[1])


def _csr(rowptr, colidx, vals, ncols, scale=None) -> Csr:
    for t, name in ((rowptr, "rowptr"), (colidx, "colidx")):
        if t.dtype != torch.int32 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous int32 tensor")
    if not vals.is_contiguous():
        raise ValueError("vals must be contiguous")
    return Csr(rowptr.numel() - 1, int(ncols), colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(vals),
               _ptr(scale), _dtype(vals))


def _dense(t: torch.Tensor, scale=None) -> Dense:
    return Dense(_ptr(t), t.shape[0], t.shape[1], _ld(t), _ptr(scale), _dtype(t))


def _opts(variant="auto", validate=False, unroll=0, ctas_per_sm=0, vecs=0) -> Opts:
    return Opts(VARIANTS[variant] if isinstance(variant, str) else int(variant), int(bool(validate)),
                int(unroll), int(ctas_per_sm), int(vecs))


def spmm_csr(rowptr, colidx, vals, B, C, M, K, N) -> None:
    """The plain FP32 entry point (legacy default stream): C = A B, Eq. 1."""
    check(lib.spmm_csr(_ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(B), _ptr(C), int(M), int(K), int(N)))


def spmm_csr_noalloc(rowptr, colidx, vals, B, C, M, K, N, stream=None) -> None:
    """FP32 SpMM (Eq. 1) that allocates nothing: the merge-path carries live in a fixed
    device array of the library (for callers that cannot allocate during a call)."""
    check(lib.spmm_csr_noalloc(_ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(B), _ptr(C), int(M), int(K), int(N),
                               _stream(stream)))


def sddmm_csr(rowptr, colidx, svals, X, Y, out, M, N, Kd) -> None:
    """The plain FP32 entry point (legacy default stream): out = S o (X Y^T), Eq. 2."""
    check(lib.sddmm_csr(_ptr(rowptr), _ptr(colidx), _ptr(svals), _ptr(X), _ptr(Y), _ptr(out), int(M), int(N),
                        int(Kd)))


def spmm(rowptr, colidx, vals, B, out=None, *, a_scale=None, b_scale=None, variant="auto", unroll=0,
         ctas_per_sm=0, vecs=0, validate=False, stream=None) -> torch.Tensor:
    """C = A B (Eq. 1) through spmm_csr_ex; returns the FP32 M x N result."""
    M = rowptr.numel() - 1
    if out is None:
        out = torch.empty((M, B.shape[1]), dtype=torch.float32, device=B.device)
    A = _csr(rowptr, colidx, vals, B.shape[0], a_scale)
    b, c = _dense(B, b_scale), _dense(out)
    o = _opts(variant, validate, unroll, ctas_per_sm, vecs)
    check(lib.spmm_csr_ex(ctypes.byref(A), ctypes.byref(b), ctypes.byref(c), ctypes.byref(o), _stream(stream)))
    return out


def sddmm(rowptr, colidx, svals, X, Y, out=None, *, x_scale=None, y_scale=None, variant="auto",
          vecs=0, validate=False, stream=None) -> torch.Tensor:
    """out[p] = s_p <X_i, Y_j> (Eq. 2) through sddmm_csr_ex; returns FP32 out[nnz]."""
    if out is None:
        out = torch.empty(colidx.numel(), dtype=torch.float32, device=X.device)
    S = _csr(rowptr, colidx, svals, Y.shape[0])
    x, y = _dense(X, x_scale), _dense(Y, y_scale)
    o = _opts(variant, validate, vecs=vecs)
    check(lib.sddmm_csr_ex(ctypes.byref(S), ctypes.byref(x), ctypes.byref(y), _ptr(out), ctypes.byref(o),
                           _stream(stream)))
    return out


def auto_choice(rowptr, ncols, colidx=None, op="spmm", b_bytes=0, row_bytes=0, stream=None) -> tuple[str, dict]:
    """The split GBSP_VARIANT_AUTO takes on this pattern for op "spmm" ('rowsplit', 'merge'
    or 'rowgroup') or "sddmm" ('rowsplit', 'merge' or 'entry'), with a gathered dense operand
    of b_bytes bytes in rows of row_bytes (0: unknown), and the row statistics it was chosen
    from (gbsp_auto_choice; a new pattern is measured at once, synchronising the stream)."""
    A = Csr(rowptr.numel() - 1, int(ncols), -1, _ptr(rowptr), _ptr(colidx) if colidx is not None else None, None,
            None, F32)
    v = ctypes.c_int32(0)
    st = (ctypes.c_int64 * 5)()
    check(lib.gbsp_auto_choice(ctypes.byref(A), {"spmm": 0, "sddmm": 1}[op], int(b_bytes), int(row_bytes),
                               _stream(stream), ctypes.byref(v), st))
    names = {k: n for n, k in VARIANTS.items()}
    keys = ("rows", "nnz", "sum_sq_lengths", "max_length", "empty_rows")
    return names[v.value], dict(zip(keys, list(st)))


def auto_forget() -> None:
    """Drops every choice GBSP_VARIANT_AUTO has kept."""
    lib.gbsp_auto_forget()


def csr_validate(rowptr, colidx, ncols, stream=None) -> int:
    """Number of CSR violations (0 for a valid matrix); synchronises the stream."""
    A = Csr(rowptr.numel() - 1, int(ncols), colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(colidx) or 1,
            None, F32)
    bad = ctypes.c_int64(0)
    st = lib.gbsp_csr_validate(ctypes.byref(A), _stream(stream), ctypes.byref(bad))
    if st not in (_lib.GBSP_OK, -2):
        check(st)
    return int(bad.value)


def quantize_bf16(x: torch.Tensor, stream=None) -> torch.Tensor:
    """bfloat16 round-to-nearest-even of an FP32 tensor (library kernel)."""
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    check(lib.gbsp_quantize_bf16(_ptr(x), _ptr(out), x.numel(), _stream(stream)))
    return out


def quantize_e4m3_rows(x: torch.Tensor, rowptr: torch.Tensor | None = None, stream=None):
    """Per-row scaled E4M3 codes (uint8) and FP32 row scales (library kernel).  Rows are
    CSR segments of the 1-D ``x`` when ``rowptr`` is given, else the rows of 2-D ``x``."""
    x = x.contiguous()
    q = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    if rowptr is None:
        nrows, ncols, ld = x.shape[0], x.shape[1], x.shape[1]
    else:
        nrows, ncols, ld = rowptr.numel() - 1, 0, 0
    scale = torch.empty(nrows, dtype=torch.float32, device=x.device)
    check(lib.gbsp_quantize_e4m3_rows(_ptr(x), _ptr(rowptr), nrows, ncols, ld, _ptr(q), _ptr(scale),
                                      _stream(stream)))
    return q, scale


def sm_count() -> int:
    return int(lib.gbsp_device_sm_count())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib.gbsp_launch_count())


class TcPlan:
    """Condensed-tile tensor-core plan of a BF16 or per-row-scaled E4M3 CSR matrix
    (gbsp_plan_create): dense 16 x 8 blocks run on tcgen05, the rest on the CSR kernels.
    ``execute(B)`` returns C = A B (E4M3: ``execute(B, row_scale=t)``)."""

    def __init__(self, rowptr, colidx, vals, ncols, threshold=0, *, row_scale=None, residual_variant="auto",
                 residual_vecs=0, residual_unroll=0, stream=None):
        self.M = rowptr.numel() - 1
        self.K = int(ncols)
        A = _csr(rowptr, colidx, vals, ncols, row_scale)
        o = _opts(residual_variant, False, residual_unroll, 0, residual_vecs)
        h = ctypes.c_void_p()
        check(lib.gbsp_plan_create(ctypes.byref(A), int(threshold), ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h

    def execute(self, B, out=None, row_scale=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.M, B.shape[1]), dtype=torch.float32, device=B.device)
        b, c = _dense(B, row_scale), _dense(out)
        check(lib.gbsp_plan_execute(self._h, ctypes.byref(b), ctypes.byref(c), _stream(stream)))
        return out

    def sddmm(self, svals, X, Y, out=None, x_scale=None, y_scale=None, tiles=-1, stream=None) -> torch.Tensor:
        """out[p] = svals[p] <X_i, Y_j> on the plan's pattern (gbsp_plan_sddmm): the dense
        blocks on tcgen05 and the rest on the CSR kernel (tiles=1), every entry on the CSR
        kernels (tiles=0), or the plan's choice (tiles=-1); returns FP32 out[nnz]."""
        if out is None:
            out = torch.empty(svals.numel(), dtype=torch.float32, device=X.device)
        x, y = _dense(X, x_scale), _dense(Y, y_scale)
        check(lib.gbsp_plan_sddmm(self._h, _ptr(svals), ctypes.byref(x), ctypes.byref(y), _ptr(out), int(tiles),
                                  _stream(stream)))
        return out

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 5)()
        check(lib.gbsp_plan_info(self._h, arr, 5))
        return {"dense_windows": arr[0], "dense_blocks": arr[1], "dense_nnz": arr[2], "residual_nnz": arr[3],
                "threshold": arr[4]}

    def check(self, stream=None) -> None:
        check(lib.gbsp_plan_check(self._h, _stream(stream)))

    def test_withhold(self, chunk: int) -> None:
        """Make the first dense window's wait for `chunk` run out (timeout-path testing)."""
        check(lib.gbsp_plan_test_withhold(self._h, int(chunk)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KbinPlan:
    """K-range-binned SpMM plan of an FP32 CSR matrix (gbsp_kbin_plan_create): A's columns
    cut into slices whose B rows stay in L2, one row-split pass per slice.  ``execute(B)``
    returns C = A B.  The plan keeps the tensors' pointers (values may change in place)."""

    def __init__(self, rowptr, colidx, vals, ncols, N=64, slice_cols=0, stream=None):
        self._keep = (rowptr, colidx, vals)
        self.M = rowptr.numel() - 1
        self.K = int(ncols)
        A = _csr(rowptr, colidx, vals, ncols)
        h = ctypes.c_void_p()
        check(lib.gbsp_kbin_plan_create(ctypes.byref(A), int(N), int(slice_cols), _stream(stream), ctypes.byref(h)))
        self._h = h

    def execute(self, B, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.M, B.shape[1]), dtype=torch.float32, device=B.device)
        b, c = _dense(B), _dense(out)
        check(lib.gbsp_kbin_plan_execute(self._h, ctypes.byref(b), ctypes.byref(c), _stream(stream)))
        return out

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 4)()
        check(lib.gbsp_kbin_plan_info(self._h, arr, 4))
        return {"slices": arr[0], "slice_cols": arr[1], "rows": arr[2], "nnz": arr[3]}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_kbin_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SellPlan:
    """SELL-C-sigma SpMM plan of an FP32 CSR matrix (gbsp_sell_plan_create): rows sorted by
    length within windows of sigma rows, slices of C rows padded and stored column-major, one
    lane group per row.  ``execute(B)`` returns C = A B.  The plan owns its copy of A."""

    def __init__(self, rowptr, colidx, vals, ncols, C=0, sigma=0, stream=None):
        self.M = rowptr.numel() - 1
        self.K = int(ncols)
        A = _csr(rowptr, colidx, vals, ncols)
        h = ctypes.c_void_p()
        check(lib.gbsp_sell_plan_create(ctypes.byref(A), int(C), int(sigma), _stream(stream), ctypes.byref(h)))
        self._h = h

    def execute(self, B, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.M, B.shape[1]), dtype=torch.float32, device=B.device)
        b, c = _dense(B), _dense(out)
        check(lib.gbsp_sell_plan_execute(self._h, ctypes.byref(b), ctypes.byref(c), _stream(stream)))
        return out

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 5)()
        check(lib.gbsp_sell_plan_info(self._h, arr, 5))
        return {"slices": arr[0], "C": arr[1], "sigma": arr[2], "slots": arr[3], "nnz": arr[4]}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_sell_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HspPlan:
    """Hyper-sparse SpMM plan of an FP32 CSR matrix (gbsp_hsp_plan_create): rows binned by
    length (long rows one warp each, short rows one lane group each, empty rows zeroed) in
    one launch.  ``execute(B)`` returns C = A B.  The plan keeps the tensors' pointers."""

    def __init__(self, rowptr, colidx, vals, ncols, stream=None):
        self._keep = (rowptr, colidx, vals)
        self.M = rowptr.numel() - 1
        self.K = int(ncols)
        A = _csr(rowptr, colidx, vals, ncols)
        h = ctypes.c_void_p()
        check(lib.gbsp_hsp_plan_create(ctypes.byref(A), _stream(stream), ctypes.byref(h)))
        self._h = h

    def execute(self, B, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.M, B.shape[1]), dtype=torch.float32, device=B.device)
        b, c = _dense(B), _dense(out)
        check(lib.gbsp_hsp_plan_execute(self._h, ctypes.byref(b), ctypes.byref(c), _stream(stream)))
        return out

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 4)()
        check(lib.gbsp_hsp_plan_info(self._h, arr, 4))
        return {"long_rows": arr[0], "short_rows": arr[1], "empty_rows": arr[2], "nnz": arr[3]}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_hsp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gnn_arrays(graphs):
    """graphs: list of (rowptr, colidx, svals, H, O, E) CUDA tensors (H, O BF16; E float32)."""
    G = len(graphs)
    S = (Csr * max(G, 1))()
    Hd = (Dense * max(G, 1))()
    Od = (Dense * max(G, 1))()
    E = (ctypes.c_void_p * max(G, 1))()
    for g, (rp, ci, sv, H, O, Ev) in enumerate(graphs):
        S[g] = _csr(rp, ci, sv, rp.numel() - 1)
        Hd[g] = _dense(H)
        Od[g] = _dense(O)
        E[g] = _ptr(Ev)
    return G, S, Hd, E, Od


class GnnPlan:
    """Batched SDDMM -> SpMM chain over many graphs as one persistent launch replayed from a
    CUDA graph (gbsp_gnn_plan_create_ex).  ``execute()`` fills every graph's E and O; with
    ``softmax=True`` each row's scores are normalised between the two products (GAT-style)
    and E receives the weights."""

    def __init__(self, graphs, edges_per_tile=0, softmax=False, stream=None):
        self._keep = graphs  # the plan holds raw pointers into these tensors
        G, S, Hd, E, Od = _gnn_arrays(graphs)
        h = ctypes.c_void_p()
        check(lib.gbsp_gnn_plan_create_ex(G, S, Hd, E, Od, int(edges_per_tile), 1 if softmax else 0, _stream(stream),
                                          ctypes.byref(h)))
        self._h = h

    def execute(self, stream=None) -> None:
        check(lib.gbsp_gnn_plan_execute(self._h, _stream(stream)))

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 4)()
        check(lib.gbsp_gnn_plan_info(self._h, arr, 4))
        return {"graphs": arr[0], "tiles": arr[1], "rows": arr[2], "edges": arr[3]}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_gnn_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gnn_sddmm_spmm_batched(graphs, stream=None) -> None:
    """One-shot batched chain (creates, runs and destroys a plan; synchronises)."""
    G, S, Hd, E, Od = _gnn_arrays(graphs)
    check(lib.gnn_sddmm_spmm_batched(G, S, Hd, E, Od, _stream(stream)))


def gnn_gat_batched(graphs, stream=None) -> None:
    """One-shot GAT-style chain: scores, row softmax into E, O = E H (synchronises)."""
    G, S, Hd, E, Od = _gnn_arrays(graphs)
    check(lib.gnn_gat_batched(G, S, Hd, E, Od, _stream(stream)))


# ---- kernel selection ------------------------------------------------------------------------

N_VARIANTS = 24
N_FEATURES = 16
N_PARAMS = 16 * 64 + 64 + 64 * 64 + 64 + 24 * 64 + 24


N_SDDMM_VARIANTS = 9
HSP_PLAN = "hsp_plan"
SELL_PLAN = "sell_plan"


def variant_options(v: int) -> dict:
    """spmm keyword arguments of selector variant v (gbsp_variant_opts); variant 23, the
    hyper-sparse plan, comes back as {"variant": "hsp_plan"} and variant 21, the SELL-C-sigma
    plan, as {"variant": "sell_plan"} (build the plan and execute it instead of calling
    spmm)."""
    o = Opts()
    check(lib.gbsp_variant_opts(int(v), ctypes.byref(o)))
    if o.variant == 6:
        return {"variant": HSP_PLAN}
    if o.variant == 7:
        return {"variant": SELL_PLAN}
    name = {1: "rowsplit", 2: "merge", 3: "scalar", 5: "rowgroup"}[o.variant]
    return {"variant": name, "vecs": o.vecs, "unroll": o.unroll, "ctas_per_sm": o.ctas_per_sm}


def sddmm_variant_options(v: int) -> dict:
    """sddmm keyword arguments of SDDMM selector variant v (gbsp_sddmm_variant_opts)."""
    o = Opts()
    check(lib.gbsp_sddmm_variant_opts(int(v), ctypes.byref(o)))
    return {"variant": {1: "rowsplit", 2: "merge", 4: "entry"}[o.variant], "vecs": o.vecs}


def features(rowptr, colidx, ncols, N, dtype=F32, out=None, stream=None) -> torch.Tensor:
    """The 16 selector features of a CSR matrix (device float32[16])."""
    if out is None:
        out = torch.empty(N_FEATURES, dtype=torch.float32, device=rowptr.device)
    A = Csr(rowptr.numel() - 1, int(ncols), colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(colidx), None, F32)
    check(lib.gbsp_features(ctypes.byref(A), int(N), int(dtype), _ptr(out), _stream(stream)))
    return out


def feature_norm(feats: torch.Tensor, stream=None) -> torch.Tensor:
    norm = torch.empty(2 * N_FEATURES, dtype=torch.float32, device=feats.device)
    check(lib.gbsp_feature_norm(_ptr(feats), feats.shape[0], _ptr(norm), _stream(stream)))
    return norm


def mlp_predict(weights, norm, feats, stream=None):
    n = feats.shape[0]
    out = torch.empty((n, N_VARIANTS), dtype=torch.float32, device=feats.device)
    choice = torch.empty(n, dtype=torch.int32, device=feats.device)
    check(lib.gbsp_mlp_predict(_ptr(weights), _ptr(norm), _ptr(feats), n, _ptr(out), _ptr(choice), _stream(stream)))
    return out, choice


def mlp_train(weights, adam, norm, feats, targets, mask, order, steps, batch=64, lr=1e-3, t0=0, stream=None):
    check(lib.gbsp_mlp_train(_ptr(weights), _ptr(adam), _ptr(norm), _ptr(feats), _ptr(targets), _ptr(mask),
                             _ptr(order), order.numel(), int(steps), int(batch), float(lr), int(t0), _stream(stream)))


def autotune(rowptr, colidx, vals, B, C, reps=3, a_scale=None, b_scale=None, stream=None):
    """Times of the 24 variants (ms, inf where not applicable) and the best index."""
    A = _csr(rowptr, colidx, vals, B.shape[0], a_scale)
    b, c = _dense(B, b_scale), _dense(C)
    times = (ctypes.c_float * N_VARIANTS)()
    best = ctypes.c_int32(-1)
    check(lib.gbsp_autotune(ctypes.byref(A), ctypes.byref(b), ctypes.byref(c), int(reps), times, ctypes.byref(best),
                            _stream(stream)))
    return [times[i] for i in range(N_VARIANTS)], best.value


def autotune_sddmm(rowptr, colidx, svals, X, Y, out, reps=3, x_scale=None, y_scale=None, stream=None):
    """Times of the SDDMM variants (ms; inf at 9..23 and where not applicable) and the best."""
    S = _csr(rowptr, colidx, svals, Y.shape[0])
    x, y = _dense(X, x_scale), _dense(Y, y_scale)
    times = (ctypes.c_float * N_VARIANTS)()
    best = ctypes.c_int32(-1)
    check(lib.gbsp_autotune_sddmm(ctypes.byref(S), ctypes.byref(x), ctypes.byref(y), _ptr(out), int(reps), times,
                                  ctypes.byref(best), _stream(stream)))
    return [times[i] for i in range(N_VARIANTS)], best.value


def _hptr(a):
    """Host address of a CPU tensor or numpy array (None for None)."""
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise ValueError("host pipeline operands live in host memory")
        return a.data_ptr() or None
    return a.ctypes.data or None


def spmm_sddmm_host(rowptr, colidx, vals, B=None, C=None, X=None, Y=None, out=None, ncols=None, chunks=8, slots=2,
                    stream=None) -> None:
    """SpMM and / or SDDMM on host-resident FP32 operands, streamed through the device in
    row chunks (gbsp_spmm_sddmm_host).  Synchronise the stream before reading C / out."""
    M = rowptr.shape[0] - 1
    nnz = colidx.shape[0]
    K = int(ncols if ncols is not None else (B.shape[0] if B is not None else Y.shape[0]))
    N = B.shape[1] if B is not None else 0
    Kd = X.shape[1] if X is not None else 0
    check(lib.gbsp_spmm_sddmm_host(_hptr(rowptr), _hptr(colidx), _hptr(vals), _hptr(B), _hptr(C), N, _hptr(X),
                                   _hptr(Y), _hptr(out), Kd, M, K, nnz, int(chunks), int(slots), _stream(stream)))


def _batch_arrays(problems, sddmm: bool):
    G = len(problems)
    A = (Csr * max(G, 1))()
    D1 = (Dense * max(G, 1))()
    D2 = (Dense * max(G, 1))()
    outs = (ctypes.c_void_p * max(G, 1))()
    for g, pr in enumerate(problems):
        if sddmm:
            rp, ci, sv, X, Y, out = pr
            A[g] = _csr(rp, ci, sv, Y.shape[0])
            D1[g], D2[g] = _dense(X), _dense(Y)
            outs[g] = _ptr(out)
        else:
            rp, ci, v, B, C = pr
            A[g] = _csr(rp, ci, v, B.shape[0])
            D1[g], D2[g] = _dense(B), _dense(C)
    return G, A, D1, D2, outs


class BatchPlan:
    """Grouped SpMM (problems: (rowptr, colidx, vals, B, C)) or SDDMM (problems:
    (rowptr, colidx, svals, X, Y, out)) over many problems in one persistent launch replayed
    from a CUDA graph."""

    def __init__(self, problems, sddmm=False, stream=None):
        self._keep = problems
        G, A, D1, D2, outs = _batch_arrays(problems, sddmm)
        h = ctypes.c_void_p()
        if sddmm:
            check(lib.gbsp_batch_plan_create_sddmm(G, A, D1, D2, outs, _stream(stream), ctypes.byref(h)))
        else:
            check(lib.gbsp_batch_plan_create_spmm(G, A, D1, D2, _stream(stream), ctypes.byref(h)))
        self._h = h

    def execute(self, stream=None) -> None:
        check(lib.gbsp_batch_plan_execute(self._h, _stream(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.gbsp_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmm_csr_batched(problems, stream=None) -> None:
    G, A, B, C, _ = _batch_arrays(problems, False)
    check(lib.spmm_csr_batched(G, A, B, C, _stream(stream)))


def sddmm_csr_batched(problems, stream=None) -> None:
    G, S, X, Y, outs = _batch_arrays(problems, True)
    check(lib.sddmm_csr_batched(G, S, X, Y, outs, _stream(stream)))


def gather_probe(table, idx, row_bytes, *, blocks=0, unroll=4, sink=None, stream=None) -> None:
    """Gather-bandwidth probe (gbsp_gather_probe): reads table[idx[p]] rows of row_bytes
    bytes with the SpMM / SDDMM lane layout and no arithmetic; time it to get the ceiling
    of the gather pattern.  ``blocks`` defaults to 8 per SM."""
    if blocks <= 0:
        blocks = 8 * sm_count()
    if sink is None or sink.numel() < blocks * 256:
        sink = torch.empty(blocks * 256, dtype=torch.int32, device=table.device)
    ld = table.stride(0) * table.element_size()
    check(lib.gbsp_gather_probe(_ptr(table), table.shape[0], int(row_bytes), int(ld), _ptr(idx), idx.numel(),
                                _ptr(sink), int(blocks), int(unroll), _stream(stream)))

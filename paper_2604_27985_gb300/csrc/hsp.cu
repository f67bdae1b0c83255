// Hyper-sparse SpMM (Eq. 1) plan: rows binned by length, several short rows per warp.
//
// Past 99.9% sparsity most rows hold a handful of entries or none, and one warp per row
// leaves most lane groups idle (a group per stored entry).  The plan reads the row lengths
// once and splits the rows into three lists: long rows (more than 32 entries) keep the
// row-split treatment (one warp per row, lane groups splitting the entries, xor-butterfly
// reduction); short rows (1 to 32 entries), sorted by length so that the groups of a warp
// finish together, get one lane group each (32 / LPN rows per warp, every group gathering
// its own row's B rows, no cross-group reduction); empty rows get their zero C rows
// stored.  A short row is a 16-byte record {row, first entry, end, first column index}
// (the pattern is fixed by the plan), so its first B gather starts right after one load.  One launch covers the three lists (consecutive block ranges, the column tile in
// blockIdx.y), so every C row is written exactly once.
#include <algorithm>
#include <vector>

#include "spmm_launch.cuh"

namespace gbsp {
namespace hsp {

using spmm_detail::gather_range;
using spmm_detail::reduce_groups;
using spmm_detail::store_row;

constexpr int kShortMax = 32;  // rows of at most this many entries take one lane group

struct HspLists {
    const int32_t *long_rows, *empty_rows;
    const int4 *short_recs;  // {row, p0, p1, colidx[p0]} per short row
    int32_t n_long, n_short, n_empty;
    int32_t b_long, b_short;  // block ranges: [0, b_long) long, then b_short short, then empty
};

// One short row per lane group: U entries at a time, every lane gathering its VPL vectors
// of each entry's B row (the group's lanes read the same index and value: one broadcast).
template <int LPN, int VPL, int U>
__device__ __forceinline__ void short_row(const SpmmProblem &P, int64_t p0, int64_t p1, int c0, int col_base,
                                          float (&acc)[VPL][4]) {
    const float4 *Bv = static_cast<const float4 *>(P.B) + col_base / 4;
    const int64_t ldv = P.ldb / 4;
    const float *vals = static_cast<const float *>(P.vals);
    bool colok[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) colok[v] = col_base + v * LPN * 4 < P.N;
    for (int64_t p = p0; p < p1; p += U) {
        int c[U];
        float a[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = p + u < p1;
            c[u] = !ok[u] ? 0 : p + u == p0 ? c0 : __ldg(P.colidx + p + u);
            a[u] = ok[u] ? __ldg(vals + p + u) : 0.f;
        }
        float4 raw[U][VPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                raw[u][v] = (ok[u] && colok[v]) ? __ldg(Bv + (int64_t)c[u] * ldv + v * LPN)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                acc[v][0] = fmaf(a[u], raw[u][v].x, acc[v][0]);
                acc[v][1] = fmaf(a[u], raw[u][v].y, acc[v][1]);
                acc[v][2] = fmaf(a[u], raw[u][v].z, acc[v][2]);
                acc[v][3] = fmaf(a[u], raw[u][v].w, acc[v][3]);
            }
    }
}

template <int LPN, int VPL, int U>
__global__ void __launch_bounds__(256) hsp_kernel(const SpmmProblem P, const HspLists L) {
    using EL = F32;
    constexpr int G = 32 / LPN;
    constexpr int TW = LPN * VPL * EL::V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col_base = blockIdx.y * TW + (lane % LPN) * EL::V;
    float acc[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
    int b = blockIdx.x;
    if (b < L.b_long) {  // one warp per long row
        const int k = b * 8 + warp;
        if (k >= L.n_long) return;
        const int row = L.long_rows[k];
        const int64_t p0 = P.rowptr[row], p1 = P.rowptr[row + 1];
        if ((blockIdx.y + 1) * TW <= P.N)
            gather_range<EL, LPN, VPL, U, false>(P, p0, p1, acc, lane, col_base);
        else
            gather_range<EL, LPN, VPL, U, true>(P, p0, p1, acc, lane, col_base);
        reduce_groups<EL, LPN, VPL>(acc);
        store_row<EL, LPN, VPL>(P.C + (int64_t)row * P.ldc, acc, lane, col_base, P.N, 1.0f);
        return;
    }
    b -= L.b_long;
    if (b < L.b_short) {  // one lane group per short row
        const int64_t k = ((int64_t)b * 8 + warp) * G + lane / LPN;
        if (k >= L.n_short) return;
        const int4 r = __ldg(L.short_recs + k);
        short_row<LPN, VPL, U>(P, r.y, r.z, r.w, col_base, acc);
        float *dst = P.C + (int64_t)r.x * P.ldc;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int col = col_base + v * LPN * EL::V;
            if (col < P.N)
                __stcs(reinterpret_cast<float4 *>(dst + col), make_float4(acc[v][0], acc[v][1], acc[v][2], acc[v][3]));
        }
        return;
    }
    b -= L.b_short;
    const int k = b * 8 + warp;  // one warp per empty row: its zero C row (this column tile)
    if (k >= L.n_empty) return;
    store_row<EL, LPN, VPL>(P.C + (int64_t)L.empty_rows[k] * P.ldc, acc, lane, col_base, P.N, 1.0f);
}

// recs[k].w = colidx[recs[k].y] (every short row has at least one entry)
__global__ void hsp_first_col_kernel(int4 *recs, int32_t n, const int32_t *colidx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        recs[k].w = colidx[recs[k].y];
}

template <int LPN, int VPL, int U>
int launch(const SpmmProblem &P, const HspLists &L, cudaStream_t s) {
    constexpr int G = 32 / LPN;
    constexpr int TW = LPN * VPL * F32::V;
    const int ntiles = (P.N + TW - 1) / TW;
    if (ntiles > 65535) return fail(GBSP_ERR_UNSUPPORTED, "hsp: N = %d needs more than 65535 column tiles", P.N);
    HspLists l = L;
    l.b_long = (L.n_long + 7) / 8;
    l.b_short = (int32_t)(((int64_t)L.n_short + 8 * G - 1) / (8 * G));
    const int64_t blocks = (int64_t)l.b_long + l.b_short + (L.n_empty + 7) / 8;
    if (blocks == 0) return ok();
    hsp_kernel<LPN, VPL, U><<<dim3((unsigned)blocks, ntiles), 256, 0, s>>>(P, l);
    count_launches(1);
    return check_launch("hsp spmm");
}

// Entries in flight per lane as in the row split: U <= LPN, VPL * U <= 16.
template <int LPN, int VPL>
int by_unroll(const SpmmProblem &P, const HspLists &L, int u, cudaStream_t s) {
    constexpr int UMAX = LPN < 16 / VPL ? LPN : 16 / VPL;
    if constexpr (UMAX >= 4) {
        if (u >= 4) return launch<LPN, VPL, 4>(P, L, s);
    }
    if constexpr (UMAX >= 2) {
        return launch<LPN, VPL, 2>(P, L, s);
    } else {
        return launch<LPN, VPL, 1>(P, L, s);
    }
}

template <int VPL>
int by_lanes(const SpmmProblem &P, const HspLists &L, int lpn, int u, cudaStream_t s) {
    switch (lpn) {
        case 1: if constexpr (VPL == 1) return by_unroll<1, 1>(P, L, u, s); break;
        case 2: if constexpr (VPL == 1) return by_unroll<2, 1>(P, L, u, s); break;
        case 4: if constexpr (VPL <= 2) return by_unroll<4, VPL>(P, L, u, s); break;
        case 8: return by_unroll<8, VPL>(P, L, u, s);
        case 16: return by_unroll<16, VPL>(P, L, u, s);
        case 32: return by_unroll<32, VPL>(P, L, u, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "hsp: no kernel for %d lanes x %d vectors", lpn, VPL);
}

}  // namespace hsp
}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::hsp;

struct gbsp_hsp_plan {
    int device;
    int64_t M, K, nnz;
    const int32_t *rowptr, *colidx;
    const float *vals;
    int32_t n_long, n_short, n_empty;
    int32_t *d_rows;  // long rows, then empty rows
    int4 *d_recs;     // short rows by decreasing length: {row, p0, p1, colidx[p0]}
};

namespace {

void hsp_free(gbsp_hsp_plan *p) {
    if (!p) return;
    cudaFree(p->d_rows);
    cudaFree(p->d_recs);
    delete p;
}

}  // namespace

GBSP_EXPORT int gbsp_hsp_plan_create(const gbsp_csr *A, void *stream, gbsp_hsp_plan **out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "hsp plan: null output");
    *out = nullptr;
    if (!A) return fail(GBSP_ERR_INVALID_ARG, "hsp plan: null matrix");
    if (A->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "hsp plan: FP32 values only");
    if (A->rows < 0 || A->cols < 0 || A->nnz < 0 || A->rows > 2147483647LL || A->cols > 2147483647LL ||
        A->nnz > 2147483647LL || (A->rows > 0 && !A->rowptr) || (A->nnz > 0 && (!A->colidx || !A->vals)))
        return fail(GBSP_ERR_INVALID_ARG, "hsp plan: bad CSR descriptor (sizes, nnz given, pointers)");
    if (A->rows == 0 && A->nnz != 0) return fail(GBSP_ERR_INVALID_CSR, "hsp plan: no rows but nnz = %lld", (long long)A->nnz);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t M = A->rows;
    std::vector<int32_t> rp((size_t)M + 1, 0);
    if (M > 0) {
        // the device check of the structure (row pointers, column range) first; then the row
        // lengths on the host
        unsigned long long *d_bad = nullptr, bad = 0;
        if (cudaMalloc(&d_bad, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(GBSP_ERR_OOM, "hsp plan: allocation failed");
        }
        int st = launch_validate(*A, d_bad, s);
        if (st == GBSP_OK &&
            (cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            st = check_launch("hsp plan validation");
        cudaFree(d_bad);
        if (st != GBSP_OK) return st;
        if (bad != 0) return fail(GBSP_ERR_INVALID_CSR, "hsp plan: %llu CSR violations", bad);
    }
    std::vector<int32_t> long_rows, empty_rows;
    std::vector<std::vector<int32_t>> by_len(kShortMax + 1);
    for (int64_t i = 0; i < M; ++i) {
        const int32_t len = rp[i + 1] - rp[i];
        if (len == 0)
            empty_rows.push_back((int32_t)i);
        else if (len > kShortMax)
            long_rows.push_back((int32_t)i);
        else
            by_len[len].push_back((int32_t)i);
    }
    std::vector<int32_t> rows(long_rows);
    rows.insert(rows.end(), empty_rows.begin(), empty_rows.end());
    std::vector<int4> recs;
    for (int len = kShortMax; len >= 1; --len)
        for (int32_t r : by_len[len]) recs.push_back(make_int4(r, rp[r], rp[r + 1], 0));
    const int32_t n_short = (int32_t)recs.size();

    gbsp_hsp_plan *p = new gbsp_hsp_plan{};
    cudaGetDevice(&p->device);
    p->M = M;
    p->K = A->cols;
    p->nnz = A->nnz;
    p->rowptr = A->rowptr;
    p->colidx = A->colidx;
    p->vals = static_cast<const float *>(A->vals);
    p->n_long = (int32_t)long_rows.size();
    p->n_short = n_short;
    p->n_empty = (int32_t)empty_rows.size();
    if (!rows.empty()) {
        if (cudaMalloc(&p->d_rows, sizeof(int32_t) * rows.size()) != cudaSuccess) {
            cudaGetLastError();
            hsp_free(p);
            return fail(GBSP_ERR_OOM, "hsp plan: allocation failed");
        }
        // stream-ordered upload: a pageable cudaMemcpy neither orders against a non-blocking
        // stream nor guarantees that the DMA has landed when it returns
        if (cudaMemcpyAsync(p->d_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            const int st = check_launch("hsp plan upload");
            hsp_free(p);
            return st ? st : fail(GBSP_ERR_CUDA, "hsp plan upload");
        }
    }
    if (!recs.empty()) {
        if (cudaMalloc(&p->d_recs, sizeof(int4) * recs.size()) != cudaSuccess) {
            cudaGetLastError();
            hsp_free(p);
            return fail(GBSP_ERR_OOM, "hsp plan: allocation failed");
        }
        if (cudaMemcpyAsync(p->d_recs, recs.data(), sizeof(int4) * recs.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            const int st = check_launch("hsp plan upload");
            hsp_free(p);
            return st ? st : fail(GBSP_ERR_CUDA, "hsp plan upload");
        }
        int64_t blocks = ((int64_t)recs.size() + 255) / 256;
        if (blocks > 32LL * sm_count()) blocks = 32LL * sm_count();
        hsp_first_col_kernel<<<(unsigned)blocks, 256, 0, s>>>(p->d_recs, n_short, p->colidx);
        count_launches(1);
        const int st = check_launch("hsp plan first columns");
        if (st != GBSP_OK) {
            cudaStreamSynchronize(s);
            hsp_free(p);
            return st;
        }
    }
    // the uploads read rows and recs, which go out of scope on return
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        const int st = check_launch("hsp plan upload");
        hsp_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "hsp plan upload");
    }
    *out = p;
    return ok();
}

GBSP_EXPORT int gbsp_hsp_plan_execute(const gbsp_hsp_plan *p, const gbsp_dense *B, gbsp_dense *C, void *stream) {
    if (!p || !B || !C) return fail(GBSP_ERR_INVALID_ARG, "hsp execute: null argument");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device)
        return fail(GBSP_ERR_INVALID_ARG, "hsp execute: plan made on device %d, current %d", p->device, dev);
    if (B->dtype != GBSP_F32 || C->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "hsp execute: FP32 B and C only");
    if (B->rows != p->K || C->rows != p->M || B->cols != C->cols || B->cols < 0 || B->ld < B->cols ||
        C->ld < C->cols || B->cols > 2147483647LL)
        return fail(GBSP_ERR_INVALID_ARG, "hsp execute: B must be K x N and C M x N (K = %lld, M = %lld)",
                    (long long)p->K, (long long)p->M);
    const int64_t N = B->cols;
    if (p->M == 0 || N == 0) return ok();
    if ((p->K > 0 && !B->data) || !C->data) return fail(GBSP_ERR_INVALID_ARG, "hsp execute: null data");
    if (N % 4 || B->ld % 4 || C->ld % 4 || !aligned16(B->data) || !aligned16(C->data))
        return fail(GBSP_ERR_ALIGN, "hsp execute: N and leading dimensions must be multiples of 4, rows "
                    "16-byte aligned");
    SpmmProblem P{};
    P.M = (int32_t)p->M;
    P.K = (int32_t)p->K;
    P.N = (int32_t)N;
    P.nnz = p->nnz;
    P.rowptr = p->rowptr;
    P.colidx = p->colidx;
    P.vals = p->vals;
    P.B = B->data;
    P.ldb = B->ld;
    P.C = static_cast<float *>(C->data);
    P.ldc = C->ld;
    P.dtype = GBSP_F32;
    HspLists L{};
    L.long_rows = p->d_rows;
    L.empty_rows = p->d_rows + p->n_long;
    L.short_recs = p->d_recs;
    L.n_long = p->n_long;
    L.n_short = p->n_short;
    L.n_empty = p->n_empty;
    int lpn, vpl;
    spmm_layout((int)(N / 4), 0, 4, lpn, vpl);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (vpl) {
        case 1: return by_lanes<1>(P, L, lpn, 4, s);
        case 2: return by_lanes<2>(P, L, lpn, 4, s);
        default: return by_lanes<4>(P, L, lpn, 4, s);
    }
}

GBSP_EXPORT int gbsp_hsp_plan_info(const gbsp_hsp_plan *p, int64_t *info, int n) {
    if (!p || !info || n < 4) return fail(GBSP_ERR_INVALID_ARG, "hsp info: need room for 4 values");
    info[0] = p->n_long;
    info[1] = p->n_short;
    info[2] = p->n_empty;
    info[3] = p->nnz;
    return ok();
}

GBSP_EXPORT void gbsp_hsp_plan_destroy(gbsp_hsp_plan *p) { hsp_free(p); }

// K-range-binned SpMM (Eq. 1) for a dense B too large for L2.
//
// The columns of A (the rows of B) are cut into S slices of W consecutive indices; pass s
// computes, for every row i, the part of C[i, :] that comes from the stored entries of row
// i with a column in slice s, so the B rows it gathers all lie in one W-row slice that
// stays resident in L2 (about 48 MB by default) while the pass runs.  Pass 0 writes C (zero
// rows where a row has nothing in the slice); each later pass adds its part to the rows
// that have entries in the slice (read, add, write of C).  This is the 1.5D idea of
// binning A's nonzeros by K-range (Section II-C: A is streamed, each processor column keeps
// one K-range of the dense operand; the routers of Section III-A filter A's entries by that
// range), with the slice held in the GPU's L2 instead of a processor's memory.
//
// Because a row's column indices are sorted, its entries in slice s are one contiguous
// range; the plan stores, per slice boundary and row, the first entry at or past that
// boundary ((S + 1) x M int32, found by binary search), and uses the caller's rowptr /
// colidx / vals in place.  Each pass is the row-split kernel's body (one warp per row,
// vectorised gathers, lane groups reduced by xor butterflies) over that range.
#include "spmm_launch.cuh"

namespace gbsp {
namespace kbin {

using spmm_detail::gather_range;
using spmm_detail::reduce_groups;
using spmm_detail::store_row;

// Counts adjacent stored entries of a row whose column indices decrease (one warp per row,
// rows striding by the grid's warps).
__global__ void __launch_bounds__(256) kbin_sorted_kernel(const int32_t *rowptr, const int32_t *colidx, int32_t M,
                                                          unsigned long long *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long count = 0;
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < M; row += nwarps) {
        const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
        for (int64_t p = p0 + lane; p + 1 < p1; p += 32)
            if (__ldg(colidx + p) > __ldg(colidx + p + 1)) ++count;
    }
    if (count) atomicAdd(bad, count);
}

// seg[b * M + i] = the first entry of row i whose column is at least b * W (b = 0..S; so
// seg[0 * M + i] = rowptr[i] and seg[S * M + i] = rowptr[i + 1]).  One thread per row.
__global__ void __launch_bounds__(256) kbin_bounds_kernel(const int32_t *rowptr, const int32_t *colidx, int32_t M,
                                                          int32_t W, int32_t S, int32_t *seg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        int32_t lo = rowptr[i];
        const int32_t end = rowptr[i + 1];
        seg[i] = lo;
        for (int32_t b = 1; b < S; ++b) {
            const int64_t target = (int64_t)b * W;
            int32_t hi = end;  // first entry in [lo, end) with colidx >= target
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (__ldg(colidx + mid) < target)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            seg[(int64_t)b * M + i] = lo;
        }
        seg[(int64_t)S * M + i] = end;
    }
}

// One pass: warp per row over the entries [lo[row], hi[row]); blockIdx.y is the column tile.
template <int LPN, int VPL, int U>
__global__ void __launch_bounds__(256) kbin_pass_kernel(const SpmmProblem P, const int32_t *__restrict__ lo,
                                                        const int32_t *__restrict__ hi, int first) {
    using EL = F32;
    constexpr int TW = LPN * VPL * EL::V;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int64_t p0 = __ldg(lo + row), p1 = __ldg(hi + row);
    if (!first && p0 == p1) return;  // nothing of this row in the slice
    const int col_base = blockIdx.y * TW + (lane % LPN) * EL::V;
    float acc[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
    if ((blockIdx.y + 1) * TW <= P.N)
        gather_range<EL, LPN, VPL, U, false>(P, p0, p1, acc, lane, col_base);
    else
        gather_range<EL, LPN, VPL, U, true>(P, p0, p1, acc, lane, col_base);
    reduce_groups<EL, LPN, VPL>(acc);
    float *dst = P.C + (int64_t)row * P.ldc;
    if (first) {
        store_row<EL, LPN, VPL>(dst, acc, lane, col_base, P.N, 1.0f);
        return;
    }
    if (lane >= LPN) return;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int col = col_base + v * LPN * EL::V;
        if (col < P.N) {
            float4 *q = reinterpret_cast<float4 *>(dst + col);
            float4 c = __ldcs(q);
            c.x += acc[v][0];
            c.y += acc[v][1];
            c.z += acc[v][2];
            c.w += acc[v][3];
            __stcs(q, c);
        }
    }
}

template <int LPN, int VPL, int U>
int launch_pass(const SpmmProblem &P, const int32_t *lo, const int32_t *hi, int first, cudaStream_t s) {
    constexpr int TW = LPN * VPL * F32::V;
    const int ntiles = (P.N + TW - 1) / TW;
    if (ntiles > 65535) return fail(GBSP_ERR_UNSUPPORTED, "kbin: N = %d needs more than 65535 column tiles", P.N);
    kbin_pass_kernel<LPN, VPL, U><<<dim3((unsigned)((P.M + 7) / 8), ntiles), 256, 0, s>>>(P, lo, hi, first);
    count_launches(1);
    return check_launch("kbin pass");
}

// Gathers in flight per lane as in the row-split SpMM: U <= LPN, VPL * U <= 16.
template <int LPN, int VPL>
int pass_unroll(const SpmmProblem &P, const int32_t *lo, const int32_t *hi, int first, int u, cudaStream_t s) {
    constexpr int UMAX = LPN < 16 / VPL ? LPN : 16 / VPL;
    if constexpr (UMAX >= 8) {
        if (u >= 8) return launch_pass<LPN, VPL, 8>(P, lo, hi, first, s);
    }
    if constexpr (UMAX >= 4) {
        if (u >= 4) return launch_pass<LPN, VPL, 4>(P, lo, hi, first, s);
    }
    if constexpr (UMAX >= 2) {
        return launch_pass<LPN, VPL, 2>(P, lo, hi, first, s);
    } else {
        return launch_pass<LPN, VPL, 1>(P, lo, hi, first, s);
    }
}

template <int VPL>
int pass_lanes(const SpmmProblem &P, const int32_t *lo, const int32_t *hi, int first, int lpn, int u,
               cudaStream_t s) {
    switch (lpn) {
        case 1: if constexpr (VPL == 1) return pass_unroll<1, 1>(P, lo, hi, first, u, s); break;
        case 2: if constexpr (VPL == 1) return pass_unroll<2, 1>(P, lo, hi, first, u, s); break;
        case 4: if constexpr (VPL <= 2) return pass_unroll<4, VPL>(P, lo, hi, first, u, s); break;
        case 8: return pass_unroll<8, VPL>(P, lo, hi, first, u, s);
        case 16: return pass_unroll<16, VPL>(P, lo, hi, first, u, s);
        case 32: return pass_unroll<32, VPL>(P, lo, hi, first, u, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "kbin: no kernel for %d lanes x %d vectors", lpn, VPL);
}

}  // namespace kbin
}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::kbin;

struct gbsp_kbin_plan {
    int device;
    int64_t M, K, nnz;
    const int32_t *rowptr, *colidx;
    const float *vals;
    int32_t W, S;
    int32_t *seg;  // (S + 1) x M
};

namespace {

constexpr int64_t kSliceBytes = 48LL << 20;  // B slice held in L2 by default
constexpr int32_t kMaxSlices = 4096;

void kbin_free(gbsp_kbin_plan *p) {
    if (!p) return;
    cudaFree(p->seg);
    delete p;
}

}  // namespace

GBSP_EXPORT int gbsp_kbin_plan_create(const gbsp_csr *A, int64_t N, int64_t slice_cols, void *stream,
                                      gbsp_kbin_plan **out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "kbin plan: null output");
    *out = nullptr;
    if (!A) return fail(GBSP_ERR_INVALID_ARG, "kbin plan: null matrix");
    if (A->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "kbin plan: FP32 values only");
    if (A->rows < 0 || A->cols < 0 || A->nnz < 0 || A->rows > 2147483647LL || A->cols > 2147483647LL ||
        A->nnz > 2147483647LL || (A->rows > 0 && !A->rowptr) || (A->nnz > 0 && (!A->colidx || !A->vals)))
        return fail(GBSP_ERR_INVALID_ARG, "kbin plan: bad CSR descriptor (sizes, nnz given, pointers)");
    if (N < 0 || slice_cols < 0) return fail(GBSP_ERR_INVALID_ARG, "kbin plan: negative N or slice width");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t M = A->rows, K = A->cols;
    int64_t W = slice_cols;
    if (W == 0) {
        const int64_t row_bytes = 4 * (N > 4 ? N : 4);
        W = kSliceBytes / row_bytes;
        if (W < 1024) W = 1024;
    }
    if (W > K) W = K > 0 ? K : 1;
    const int64_t S = K > 0 ? (K + W - 1) / W : 1;
    if (S > kMaxSlices)
        return fail(GBSP_ERR_INVALID_ARG, "kbin plan: %lld slices of %lld columns exceed %d", (long long)S,
                    (long long)W, kMaxSlices);
    // structure first (rowptr, column range); rows are walked only once it holds.  Then the
    // rows must be sorted, so that each row's entries in a slice form one range.
    if (M == 0 && A->nnz != 0) return fail(GBSP_ERR_INVALID_CSR, "kbin plan: no rows but nnz = %lld", (long long)A->nnz);
    unsigned long long *d_bad = nullptr;
    if (M > 0 && cudaMalloc(&d_bad, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBSP_ERR_OOM, "kbin plan: allocation failed");
    }
    int st = M > 0 ? launch_validate(*A, d_bad, s) : GBSP_OK;
    unsigned long long bad[2] = {0, 0};
    if (st == GBSP_OK && M > 0 && cudaMemsetAsync(d_bad + 1, 0, sizeof(unsigned long long), s) != cudaSuccess)
        st = check_launch("kbin plan memset");
    if (st == GBSP_OK && M > 0 &&
        (cudaMemcpyAsync(bad, d_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        st = check_launch("kbin plan validation");
    if (st == GBSP_OK && bad[0] != 0) st = fail(GBSP_ERR_INVALID_CSR, "kbin plan: %llu CSR violations", bad[0]);
    if (st == GBSP_OK && M > 0) {
        int64_t blocks = (M + 7) / 8;
        if (blocks > 16LL * sm_count()) blocks = 16LL * sm_count();
        kbin_sorted_kernel<<<(unsigned)blocks, 256, 0, s>>>(A->rowptr, A->colidx, (int32_t)M, d_bad + 1);
        count_launches(1);
        if (cudaMemcpyAsync(bad + 1, d_bad + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = check_launch("kbin plan sorted check");
        else if (bad[1] != 0)
            st = fail(GBSP_ERR_INVALID_CSR, "kbin plan: column indices must not decrease within a row "
                      "(%llu places do)", bad[1]);
    }
    cudaFree(d_bad);
    if (st != GBSP_OK) return st;

    gbsp_kbin_plan *p = new gbsp_kbin_plan{};
    cudaGetDevice(&p->device);
    p->M = M;
    p->K = K;
    p->nnz = A->nnz;
    p->rowptr = A->rowptr;
    p->colidx = A->colidx;
    p->vals = static_cast<const float *>(A->vals);
    p->W = (int32_t)W;
    p->S = (int32_t)S;
    if (M > 0) {
        if (cudaMalloc(&p->seg, sizeof(int32_t) * (size_t)(S + 1) * (size_t)M) != cudaSuccess) {
            cudaGetLastError();
            kbin_free(p);
            return fail(GBSP_ERR_OOM, "kbin plan: %lld x %lld slice offsets do not fit", (long long)(S + 1),
                        (long long)M);
        }
        int64_t blocks = (M + 255) / 256;
        if (blocks > 32LL * sm_count()) blocks = 32LL * sm_count();
        kbin_bounds_kernel<<<(unsigned)blocks, 256, 0, s>>>(A->rowptr, A->colidx, (int32_t)M, p->W, p->S, p->seg);
        count_launches(1);
        st = check_launch("kbin plan bounds");
        if (st != GBSP_OK) {
            kbin_free(p);
            return st;
        }
    }
    *out = p;
    return ok();
}

GBSP_EXPORT int gbsp_kbin_plan_execute(const gbsp_kbin_plan *p, const gbsp_dense *B, gbsp_dense *C, void *stream) {
    if (!p || !B || !C) return fail(GBSP_ERR_INVALID_ARG, "kbin execute: null argument");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) return fail(GBSP_ERR_INVALID_ARG, "kbin execute: plan made on device %d, current %d",
                                      p->device, dev);
    if (B->dtype != GBSP_F32 || C->dtype != GBSP_F32)
        return fail(GBSP_ERR_UNSUPPORTED, "kbin execute: FP32 B and C only");
    if (B->rows != p->K || C->rows != p->M || B->cols != C->cols || B->cols < 0 || B->ld < B->cols ||
        C->ld < C->cols || B->cols > 2147483647LL)
        return fail(GBSP_ERR_INVALID_ARG, "kbin execute: B must be K x N and C M x N (K = %lld, M = %lld)",
                    (long long)p->K, (long long)p->M);
    const int64_t N = B->cols;
    if (p->M == 0 || N == 0) return ok();
    if ((p->K > 0 && !B->data) || !C->data) return fail(GBSP_ERR_INVALID_ARG, "kbin execute: null data");
    if (N % 4 || B->ld % 4 || C->ld % 4 || !aligned16(B->data) || !aligned16(C->data))
        return fail(GBSP_ERR_ALIGN, "kbin execute: N and leading dimensions must be multiples of 4, rows "
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
    int lpn, vpl;
    spmm_layout((int)(N / 4), 0, 4, lpn, vpl);
    const int u = vpl == 1 ? 8 : 4;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int32_t b = 0; b < p->S; ++b) {
        const int32_t *lo = p->seg + (int64_t)b * p->M, *hi = p->seg + (int64_t)(b + 1) * p->M;
        const int first = b == 0;
        int st;
        switch (vpl) {
            case 1: st = pass_lanes<1>(P, lo, hi, first, lpn, u, s); break;
            case 2: st = pass_lanes<2>(P, lo, hi, first, lpn, u, s); break;
            default: st = pass_lanes<4>(P, lo, hi, first, lpn, u, s); break;
        }
        if (st != GBSP_OK) return st;
    }
    return ok();
}

GBSP_EXPORT int gbsp_kbin_plan_info(const gbsp_kbin_plan *p, int64_t *info, int n) {
    if (!p || !info || n < 4) return fail(GBSP_ERR_INVALID_ARG, "kbin info: need room for 4 values");
    info[0] = p->S;
    info[1] = p->W;
    info[2] = p->M;
    info[3] = p->nnz;
    return ok();
}

GBSP_EXPORT void gbsp_kbin_plan_destroy(gbsp_kbin_plan *p) { kbin_free(p); }

// SpMM (Eq. 1) through SELL-C-sigma: the padded sliced format the paper's own design builds
// on (its SELLPACK-like stream, Section III-A) and names among the formats to explore
// (Section V), laid out for this GPU.
//
// Rows are sorted by decreasing length within windows of sigma consecutive rows, then cut
// into slices of C rows; each slice is padded to its longest row and stored column-major,
// so entry j of the slice's row r sits at slice_off[s] + j * C + r.  One lane group of LPN
// lanes takes one row (as in the row groups), several rows per warp: at each step the
// groups of a block read consecutive slots (one coalesced index load for 8 * G rows), and
// the rows of a warp have about the same length (they were sorted), so its groups finish
// together.  Padding slots are never read: every group stops at its own row's length.
// A long row keeps its group busy alone, the format's known weak spot on skewed rows.
#include <algorithm>
#include <numeric>
#include <vector>

#include "spmm_launch.cuh"

namespace gbsp {
namespace sell {

struct SellView {
    const int32_t *perm, *len;   // per sorted position: original row, length
    const int64_t *slice_off;    // per slice: first slot
    const int32_t *colidx;       // slots
    const float *vals;
    int32_t nrows, C;            // sorted positions (= M), slice height
};

template <int LPN, int VPL, int U>
__global__ void __launch_bounds__(256) sell_kernel(const SpmmProblem P, const SellView S, int blocks_per_slice) {
    constexpr int G = 32 / LPN;
    constexpr int TW = LPN * VPL * 4;
    const int lane = threadIdx.x & 31;
    const int slice = blockIdx.x / blocks_per_slice;
    const int r_local = (blockIdx.x % blocks_per_slice) * 8 * G + (threadIdx.x >> 5) * G + lane / LPN;
    const int64_t r = (int64_t)slice * S.C + r_local;
    if (r >= S.nrows) return;  // a group's lanes share r; no warp-wide exchange follows
    const int row = __ldg(S.perm + r), L = __ldg(S.len + r);
    const int64_t base = __ldg(S.slice_off + slice) + r_local;
    const int col_base = blockIdx.y * TW + (lane % LPN) * 4;
    const float4 *Bv = static_cast<const float4 *>(P.B) + col_base / 4;
    const int64_t ldv = P.ldb / 4;
    bool colok[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) colok[v] = col_base + v * LPN * 4 < P.N;
    float acc[VPL][4];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v][0] = acc[v][1] = acc[v][2] = acc[v][3] = 0.f;
    for (int j = 0; j < L; j += U) {
        int c[U];
        float a[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = j + u < L;
            const int64_t slot = base + (int64_t)(j + u) * S.C;
            c[u] = ok[u] ? ld_stream(S.colidx + slot) : 0;
            a[u] = ok[u] ? ld_stream(S.vals + slot) : 0.f;
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
    float *dst = P.C + (int64_t)row * P.ldc;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int col = col_base + v * LPN * 4;
        if (col < P.N)
            __stcs(reinterpret_cast<float4 *>(dst + col), make_float4(acc[v][0], acc[v][1], acc[v][2], acc[v][3]));
    }
}

// One warp per sorted position: its row's entries go to their column-major slots.
__global__ void sell_fill_kernel(const int32_t *rowptr, const int32_t *colidx, const float *vals, SellView S,
                                 int32_t *out_col, float *out_val) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < S.nrows; r += warps) {
        const int row = S.perm[r];
        const int64_t p0 = rowptr[row], L = rowptr[row + 1] - p0;
        const int64_t slice = r / S.C;
        const int64_t base = S.slice_off[slice] + (r - slice * S.C);
        for (int64_t j = lane; j < L; j += 32) {
            out_col[base + j * S.C] = colidx[p0 + j];
            out_val[base + j * S.C] = vals[p0 + j];
        }
    }
}

template <int LPN, int VPL, int U>
int launch(const SpmmProblem &P, const SellView &S, cudaStream_t s) {
    constexpr int G = 32 / LPN;
    constexpr int TW = LPN * VPL * 4;
    if (S.C % (8 * G)) return fail(GBSP_ERR_UNSUPPORTED, "sell: C = %d is not a multiple of %d rows", S.C, 8 * G);
    const int bps = S.C / (8 * G);
    const int64_t nslices = ((int64_t)S.nrows + S.C - 1) / S.C;
    const int ntiles = (P.N + TW - 1) / TW;
    if (nslices * bps > 2147483647LL || ntiles > 65535) return fail(GBSP_ERR_UNSUPPORTED, "sell: grid too large");
    if (nslices == 0) return ok();
    sell_kernel<LPN, VPL, U><<<dim3((unsigned)(nslices * bps), ntiles), 256, 0, s>>>(P, S, bps);
    count_launches(1);
    return check_launch("sell spmm");
}

template <int VPL>
int by_lanes(const SpmmProblem &P, const SellView &S, int lpn, cudaStream_t s) {
    switch (lpn) {
        case 1: if constexpr (VPL == 1) return launch<1, 1, 4>(P, S, s); break;
        case 2: if constexpr (VPL == 1) return launch<2, 1, 4>(P, S, s); break;
        case 4: if constexpr (VPL <= 2) return launch<4, VPL, 4>(P, S, s); break;
        case 8: return launch<8, VPL, 4>(P, S, s);
        case 16: return launch<16, VPL, 4>(P, S, s);
        case 32: return launch<32, VPL, 4>(P, S, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "sell: no kernel for %d lanes x %d vectors", lpn, VPL);
}

}  // namespace sell
}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::sell;

struct gbsp_sell_plan {
    int device;
    int64_t M, K, nnz, slots, nslices;
    int32_t C, sigma;
    int32_t *perm, *len, *colidx;
    int64_t *slice_off;
    float *vals;
};

namespace {
void sell_free(gbsp_sell_plan *p) {
    if (!p) return;
    cudaFree(p->perm);
    cudaFree(p->len);
    cudaFree(p->slice_off);
    cudaFree(p->colidx);
    cudaFree(p->vals);
    delete p;
}
}  // namespace

GBSP_EXPORT int gbsp_sell_plan_create(const gbsp_csr *A, int32_t C, int32_t sigma, void *stream,
                                      gbsp_sell_plan **out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "sell plan: null output");
    *out = nullptr;
    if (!A || A->rows < 0 || A->cols < 0 || A->rows > 2147483647LL || A->cols > 2147483647LL || A->nnz < 0 ||
        (A->rows > 0 && !A->rowptr) || (A->nnz > 0 && (!A->colidx || !A->vals)))
        return fail(GBSP_ERR_INVALID_ARG, "sell plan: bad CSR (nnz must be given)");
    if (A->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "sell plan: FP32 values only");
    if (C <= 0) C = 64;
    if (C % 8 || C > 1024) return fail(GBSP_ERR_INVALID_ARG, "sell plan: C must be a multiple of 8, at most 1024");
    const int64_t M = A->rows;
    if (sigma <= 0 || sigma > M) sigma = (int32_t)(M > 0 ? M : 1);
    if (sigma % C && sigma != M) return fail(GBSP_ERR_INVALID_ARG, "sell plan: sigma must be a multiple of C");
    int64_t bad = 0;
    int st = gbsp_csr_validate(A, stream, &bad);  // synchronises the stream
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> rp(M + 1);
    if (M > 0 && (cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int32_t) * (M + 1), cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess))
        return check_launch("sell plan: read rowptr");
    // sort by decreasing length within windows of sigma rows (stable: ties keep row order)
    std::vector<int32_t> perm(M), len(M);
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t w0 = 0; w0 < M; w0 += sigma) {
        const int64_t w1 = std::min<int64_t>(M, w0 + sigma);
        std::stable_sort(perm.begin() + w0, perm.begin() + w1,
                         [&](int32_t a, int32_t b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
    }
    for (int64_t r = 0; r < M; ++r) len[r] = rp[perm[r] + 1] - rp[perm[r]];
    const int64_t nslices = (M + C - 1) / C;
    std::vector<int64_t> off(nslices + 1, 0);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int32_t mx = 0;
        for (int64_t r = sl * C; r < std::min<int64_t>(M, (sl + 1) * C); ++r) mx = std::max(mx, len[r]);
        off[sl + 1] = off[sl] + (int64_t)mx * C;
    }
    gbsp_sell_plan *p = new gbsp_sell_plan{};
    cudaGetDevice(&p->device);
    p->M = M;
    p->K = A->cols;
    p->nnz = A->nnz;
    p->C = C;
    p->sigma = sigma;
    p->nslices = nslices;
    p->slots = off[nslices];
    if (cudaMalloc(&p->perm, sizeof(int32_t) * (M ? M : 1)) != cudaSuccess ||
        cudaMalloc(&p->len, sizeof(int32_t) * (M ? M : 1)) != cudaSuccess ||
        cudaMalloc(&p->slice_off, sizeof(int64_t) * (nslices + 1)) != cudaSuccess ||
        cudaMalloc(&p->colidx, sizeof(int32_t) * (p->slots ? p->slots : 1)) != cudaSuccess ||
        cudaMalloc(&p->vals, sizeof(float) * (p->slots ? p->slots : 1)) != cudaSuccess) {
        cudaGetLastError();
        sell_free(p);
        return fail(GBSP_ERR_OOM, "sell plan: allocation failed (%lld slots)", (long long)off[nslices]);
    }
    // stream-ordered uploads, complete before the host vectors go out of scope
    if ((M && (cudaMemcpyAsync(p->perm, perm.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemcpyAsync(p->len, len.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice, s) != cudaSuccess)) ||
        cudaMemcpyAsync(p->slice_off, off.data(), sizeof(int64_t) * (nslices + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
        st = check_launch("sell plan upload");
        cudaStreamSynchronize(s);
        sell_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "sell plan upload");
    }
    if (M > 0 && p->nnz > 0) {
        SellView v{p->perm, p->len, p->slice_off, p->colidx, p->vals, (int32_t)M, C};
        int64_t blocks = (M + 7) / 8;
        if (blocks > 32LL * sm_count()) blocks = 32LL * sm_count();
        sell_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(A->rowptr, A->colidx, static_cast<const float *>(A->vals), v,
                                                         p->colidx, p->vals);
        count_launches(1);
        st = check_launch("sell plan fill");
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = check_launch("sell plan fill");
    if (st) {
        sell_free(p);
        return st;
    }
    *out = p;
    return ok();
}

GBSP_EXPORT int gbsp_sell_plan_execute(const gbsp_sell_plan *p, const gbsp_dense *B, gbsp_dense *Cd, void *stream) {
    if (!p || !B || !Cd) return fail(GBSP_ERR_INVALID_ARG, "sell execute: null argument");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) return fail(GBSP_ERR_INVALID_ARG, "sell execute: the current device is not the plan's");
    if (B->dtype != GBSP_F32 || Cd->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "sell execute: FP32 only");
    if (B->rows != p->K || Cd->rows != p->M || Cd->cols != B->cols || B->ld < B->cols || Cd->ld < Cd->cols ||
        (B->rows > 0 && B->cols > 0 && !B->data) || (Cd->rows > 0 && Cd->cols > 0 && !Cd->data))
        return fail(GBSP_ERR_INVALID_ARG, "sell execute: shape mismatch");
    if (B->cols % 4 || B->ld % 4 || Cd->ld % 4 || !aligned16(B->data) || !aligned16(Cd->data))
        return fail(GBSP_ERR_ALIGN, "sell execute: N and both ld multiples of 4, B and C 16-byte aligned");
    if (p->M == 0 || B->cols == 0) return ok();
    SpmmProblem P{};
    P.M = (int32_t)p->M;
    P.K = (int32_t)p->K;
    P.N = (int32_t)B->cols;
    P.nnz = p->nnz;
    P.B = B->data;
    P.ldb = B->ld;
    P.C = static_cast<float *>(Cd->data);
    P.ldc = Cd->ld;
    P.dtype = GBSP_F32;
    SellView v{p->perm, p->len, p->slice_off, p->colidx, p->vals, (int32_t)p->M, p->C};
    int lpn, vpl;
    spmm_layout(P.N / 4, 0, 4, lpn, vpl);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st;
    switch (vpl) {
        case 1: st = by_lanes<1>(P, v, lpn, s); break;
        case 2: st = by_lanes<2>(P, v, lpn, s); break;
        default: st = by_lanes<4>(P, v, lpn, s); break;
    }
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_sell_plan_info(const gbsp_sell_plan *p, int64_t *info, int n) {
    if (!p || !info) return fail(GBSP_ERR_INVALID_ARG, "sell info: null argument");
    const int64_t v[5] = {p->nslices, p->C, p->sigma, p->slots, p->nnz};
    for (int k = 0; k < n && k < 5; ++k) info[k] = v[k];
    return ok();
}

GBSP_EXPORT void gbsp_sell_plan_destroy(gbsp_sell_plan *p) { sell_free(p); }

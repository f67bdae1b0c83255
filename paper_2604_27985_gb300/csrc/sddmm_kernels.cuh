// SDDMM kernels (Eq. 2): out[p] = s_p * <X_i, Y_colidx[p]> for every stored entry p of row i.
//
// One warp per row of S.  The row's X_i is held in registers for the whole row.  The warp
// splits into G = 32 / LPN groups of LPN lanes; each lane covers VPL 16-byte vectors of the
// Kd-long rows.  Entries are taken 32 at a time: at step t (0 <= t < LPN) group g gathers
// Y_j of entry g * LPN + t and each lane keeps its partial dot in part[t].  After the LPN
// steps a reduce-scatter across the group (log2 LPN exchange rounds, halving the values
// each round) leaves lane g * LPN + sl with the complete dot of entry g * LPN + sl, i.e.
// lane L holds entry L of the chunk, so the results leave in one coalesced store.
#pragma once

#include "common.cuh"

namespace gbsp {
namespace sddmm_detail {

// Partial dots of one chunk: part[t] is this lane's share of the dot of entry g * LPN + t.
template <class EL, int LPN, int VPL, bool CHECK_COLS, bool CHECK_NNZ>
__device__ __forceinline__ void sddmm_chunk(const uint4 *__restrict__ Yv, int64_t ldv, int c, int cnt, int g,
                                            const bool (&colok)[VPL], const float (&x)[VPL][EL::V],
                                            float (&part)[LPN]) {
#pragma unroll
    for (int t = 0; t < LPN; ++t) part[t] = 0.f;
#pragma unroll
    for (int t = 0; t < LPN; ++t) {
        if (CHECK_NNZ && t >= cnt) break;  // no group has an entry at this step (warp-uniform)
        const int idx = g * LPN + t;
        const int cj = __shfl_sync(FULL, c, idx);
        const uint4 *rp = Yv + (int64_t)cj * ldv;
        uint4 raw[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            if constexpr (CHECK_COLS || CHECK_NNZ) {
                bool ok = true;
                if constexpr (CHECK_NNZ) ok = idx < cnt;
                if constexpr (CHECK_COLS) ok = ok && colok[v];
                raw[v] = ok ? ld_gather16(rp + v * LPN) : make_uint4(0, 0, 0, 0);
            } else {
                raw[v] = ld_gather16(rp + v * LPN);
            }
        }
        float sum = 0.f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            float y[EL::V];
            EL::unpack(raw[v], y);
#pragma unroll
            for (int k = 0; k < EL::V; ++k) sum = fmaf(x[v][k], y[k], sum);
        }
        part[t] = sum;
    }
}

// Entries [p0, p1) of row `row`: X_i in registers, entries 32 at a time with the next 32
// column indices and values prefetched while the current ones are used.
template <class EL, int LPN, int VPL, bool CHECK_COLS>
__device__ __forceinline__ void sddmm_segment(const SddmmProblem &P, int row, int64_t p0, int64_t p1, int lane) {
    const int sl = lane % LPN, g = lane / LPN;
    using ST = typename EL::stored;
    const ST *X = static_cast<const ST *>(P.X);
    const uint4 *Yv = static_cast<const uint4 *>(P.Y) + sl;
    const int64_t ldv = P.ldy / EL::V;

    bool colok[VPL];
    float x[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int k0 = (v * LPN + sl) * EL::V;
        colok[v] = !CHECK_COLS || k0 < P.Kd;
        uint4 raw = make_uint4(0, 0, 0, 0);
        if (colok[v]) raw = ld_gather16(X + (int64_t)row * P.ldx + k0);
        EL::unpack(raw, x[v]);
    }
    const float xs = EL::dtype == GBSP_E4M3 ? __ldg(P.x_scale + row) : 1.0f;

    int c = 0;
    float s = 0.f;
    if (p0 + lane < p1) {
        c = ld_stream(P.colidx + p0 + lane);
        s = ld_stream(P.svals + p0 + lane);
    }
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t nb = base + 32;
        int c2 = 0;
        float s2 = 0.f;
        if (nb + lane < p1) {
            c2 = ld_stream(P.colidx + nb + lane);
            s2 = ld_stream(P.svals + nb + lane);
        }
        float part[LPN];
        if (nb <= p1)
            sddmm_chunk<EL, LPN, VPL, CHECK_COLS, false>(Yv, ldv, c, 32, g, colok, x, part);
        else
            sddmm_chunk<EL, LPN, VPL, CHECK_COLS, true>(Yv, ldv, c, (int)(p1 - base), g, colok, x, part);
#pragma unroll
        for (int h = LPN / 2; h >= 1; h >>= 1) {
            const bool upper = (sl & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = upper ? part[i] : part[i + h];
                const float keep = upper ? part[i + h] : part[i];
                part[i] = keep + __shfl_xor_sync(FULL, send, h);
            }
        }
        if (base + lane < p1) {
            float r = s * part[0];
            if (EL::dtype == GBSP_E4M3) r *= xs * __ldg(P.y_scale + c);
            __stcs(P.out + base + lane, r);
        }
        c = c2;
        s = s2;
    }
}

// One warp per row of S.
template <class EL, int LPN, int VPL>
__global__ void __launch_bounds__(256) sddmm_rowsplit_kernel(const SddmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    if (P.Kd == LPN * VPL * EL::V)
        sddmm_segment<EL, LPN, VPL, false>(P, row, p0, p1, lane);
    else
        sddmm_segment<EL, LPN, VPL, true>(P, row, p0, p1, lane);
}

// nnz-balanced split: warp w takes the items [w * ipw, (w + 1) * ipw) of the merge path
// over (row ends, stored entries) and computes every entry in it, row segment by row
// segment.  Each output belongs to one entry, so no carries are needed.
template <class EL, int LPN, int VPL>
__global__ void __launch_bounds__(256) sddmm_merge_kernel(const SddmmProblem P, int nwarps) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nnz = __ldg(P.rowptr + P.M);
    const int64_t total = (int64_t)P.M + nnz;
    const int64_t ipw = (total + nwarps - 1) / nwarps;
    const int64_t d0 = min((int64_t)w * ipw, total);
    const int64_t d1 = min(d0 + ipw, total);
    const int x0 = merge_search(P.rowptr, P.M, nnz, d0, lane);
    const int x1 = merge_search(P.rowptr, P.M, nnz, d1, lane);
    int64_t p = d0 - x0;
    const int64_t y1 = d1 - x1;
    const bool full = P.Kd == LPN * VPL * EL::V;
    for (int row = x0; row <= x1 && row < P.M; ++row) {
        const int64_t e = row < x1 ? (int64_t)__ldg(P.rowptr + row + 1) : y1;
        if (e > p) {
            if (full)
                sddmm_segment<EL, LPN, VPL, false>(P, row, p, e, lane);
            else
                sddmm_segment<EL, LPN, VPL, true>(P, row, p, e, lane);
        }
        p = e;
    }
}

// Any Kd and alignment: one lane per stored entry, plain loads.  X_i is read by all lanes
// of the warp at the same address (a broadcast).  Suits small Kd such as the paper's D = 2.
template <class EL>
__global__ void __launch_bounds__(256) sddmm_scalar_kernel(const SddmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    using ST = typename EL::stored;
    const ST *X = static_cast<const ST *>(P.X) + (int64_t)row * P.ldx;
    const ST *Y = static_cast<const ST *>(P.Y);
    const float xs = EL::dtype == GBSP_E4M3 ? __ldg(P.x_scale + row) : 1.0f;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        const int c = ld_stream(P.colidx + p);
        const ST *y = Y + (int64_t)c * P.ldy;
        float sum = 0.f;
        for (int k = 0; k < P.Kd; ++k) sum = fmaf(EL::scalar(X + k), EL::scalar(y + k), sum);
        float r = ld_stream(P.svals + p) * sum;
        if (EL::dtype == GBSP_E4M3) r *= xs * __ldg(P.y_scale + c);
        P.out[p] = r;
    }
}

}  // namespace sddmm_detail

}  // namespace gbsp

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
// PAIR (VPL = 2, full rows only): the lane's two vectors are adjacent and arrive by one
// 32-byte load.
template <class EL, int LPN, int VPL, bool CHECK_COLS, bool CHECK_NNZ, bool PAIR = false>
__device__ __forceinline__ void sddmm_chunk(const uint4 *__restrict__ Yv, int64_t ldv, int c, int cnt, int g,
                                            const bool (&colok)[VPL], const uint4 (&xr)[VPL],
                                            const float (&x)[VPL][EL::V], float (&part)[LPN]) {
    static_assert(!PAIR || (VPL == 2 && !CHECK_COLS), "paired loads cover whole rows of two vectors per lane");
#pragma unroll
    for (int t = 0; t < LPN; ++t) part[t] = 0.f;
#pragma unroll
    for (int t = 0; t < LPN; ++t) {
        if (CHECK_NNZ && t >= cnt) break;  // no group has an entry at this step (warp-uniform)
        const int idx = g * LPN + t;
        const int cj = __shfl_sync(FULL, c, idx);
        const uint4 *rp = Yv + (int64_t)cj * ldv;
        uint4 raw[VPL];
        if constexpr (PAIR) {
            if (!CHECK_NNZ || idx < cnt) {
                ld_gather32(rp, raw[0], raw[VPL - 1]);
            } else {
                raw[0] = make_uint4(0, 0, 0, 0);
                raw[VPL - 1] = raw[0];
            }
        } else
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
        for (int v = 0; v < VPL; ++v) sum = EL::dot(xr[v], x[v], raw[v], sum);
        part[t] = sum;
    }
}

// Entries [p0, p1) of row `row`: X_i in registers, entries 32 at a time with the next 32
// column indices and values prefetched while the current ones are used.  With POS, entry
// e's value and output sit at position P.pos[e] of the caller's arrays (a sub-matrix of
// another CSR, such as the residual of a tensor-core plan).
template <class EL, int LPN, int VPL, bool CHECK_COLS, bool POS = false, bool PAIR = false>
__device__ __forceinline__ void sddmm_segment(const SddmmProblem &P, int row, int64_t p0, int64_t p1, int lane) {
    const int sl = lane % LPN, g = lane / LPN;
    using ST = typename EL::stored;
    const ST *X = static_cast<const ST *>(P.X);
    // a lane's vectors: v * LPN + sl (each instruction of a group reads one contiguous span),
    // or 2 * sl + v when paired (one 32-byte load per lane)
    const uint4 *Yv = static_cast<const uint4 *>(P.Y) + (PAIR ? 2 * sl : sl);
    const int64_t ldv = P.ldy / EL::V;

    bool colok[VPL];
    uint4 xr[VPL];
    float x[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int k0 = (PAIR ? 2 * sl + v : v * LPN + sl) * EL::V;
        colok[v] = !CHECK_COLS || k0 < P.Kd;
        xr[v] = make_uint4(0, 0, 0, 0);
        if (colok[v]) xr[v] = ld_gather16(X + (int64_t)row * P.ldx + k0);
        EL::unpack(xr[v], x[v]);
    }
    const float xs = EL::dtype == GBSP_E4M3 ? __ldg(P.x_scale + row) : 1.0f;

    int c = 0;
    float s = 0.f;
    int64_t q = p0 + lane;  // where this lane's entry keeps its value and output
    if (p0 + lane < p1) {
        c = ld_stream(P.colidx + p0 + lane);
        if constexpr (POS) q = __ldg(P.pos + p0 + lane);
        s = ld_stream(P.svals + q);
    }
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t nb = base + 32;
        int c2 = 0;
        float s2 = 0.f;
        int64_t q2 = nb + lane;
        if (nb + lane < p1) {
            c2 = ld_stream(P.colidx + nb + lane);
            if constexpr (POS) q2 = __ldg(P.pos + nb + lane);
            s2 = ld_stream(P.svals + q2);
        }
        float part[LPN];
        if (nb <= p1)
            sddmm_chunk<EL, LPN, VPL, CHECK_COLS, false, PAIR>(Yv, ldv, c, 32, g, colok, xr, x, part);
        else
            sddmm_chunk<EL, LPN, VPL, CHECK_COLS, true, PAIR>(Yv, ldv, c, (int)(p1 - base), g, colok, xr, x, part);
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
            __stcs(P.out + (POS ? q : base + lane), r);
        }
        c = c2;
        if constexpr (POS) q = q2;
        s = s2;
    }
}

// One warp per row of S.  PAIR requires Kd = LPN * 2 * V with 32-byte aligned rows of X and Y
// (the launcher checks).
template <class EL, int LPN, int VPL, bool POS = false, bool PAIR = false>
__global__ void __launch_bounds__(256) sddmm_rowsplit_kernel(const SddmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    if constexpr (PAIR) {
        sddmm_segment<EL, LPN, VPL, false, POS, true>(P, row, p0, p1, lane);
    } else {
        if (P.Kd == LPN * VPL * EL::V)
            sddmm_segment<EL, LPN, VPL, false, POS>(P, row, p0, p1, lane);
        else
            sddmm_segment<EL, LPN, VPL, true, POS>(P, row, p0, p1, lane);
    }
}

// nnz-balanced split: warp w takes the items [w * ipw, (w + 1) * ipw) of the merge path
// over (row ends, stored entries) and computes every entry in it, row segment by row
// segment.  Each output belongs to one entry, so no carries are needed.
template <class EL, int LPN, int VPL, bool PAIR = false>
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
            if constexpr (PAIR)
                sddmm_segment<EL, LPN, VPL, false, false, true>(P, row, p, e, lane);
            else if (full)
                sddmm_segment<EL, LPN, VPL, false>(P, row, p, e, lane);
            else
                sddmm_segment<EL, LPN, VPL, true>(P, row, p, e, lane);
        }
        p = e;
    }
}

// ---- entry split ------------------------------------------------------------------------
//
// For short or skewed rows: a warp takes a range of stored entries regardless of row
// boundaries, 32 at a time, so no lane idles at the end of a short row and no warp waits
// on a row's start.  Each chunk finds the row of every lane's entry from the row pointers
// (one coalesced load of 32 row ends, then a 6-step binary search across the lanes by
// shuffles), and a lane group reloads X_i only when the row of its entry changes.

// Number of rows whose last entry precedes entry e (the row holding e): a 33-ary
// warp-cooperative search over the row ends rowptr[1..M].
__device__ __forceinline__ int row_of_entry(const int32_t *rowptr, int M, int64_t e, int lane) {
    int64_t lo = 0, hi = M;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t span = hi - lo;
        const int64_t probe = lo + (span * (lane + 1)) / 33;
        const bool t = (int64_t)__ldg(rowptr + probe + 1) <= e;
        const int k = __popc(__ballot_sync(FULL, t));
        const int64_t new_lo = k == 0 ? lo : lo + (span * k) / 33 + 1;
        const int64_t new_hi = k == 32 ? hi : lo + (span * (k + 1)) / 33;
        lo = new_lo;
        hi = new_hi;
    }
    const int64_t x = lo + lane;
    const bool t = x < hi && (int64_t)__ldg(rowptr + x + 1) <= e;
    return (int)(lo + __popc(__ballot_sync(FULL, t)));
}

// End of row rb + lane (rows past M end at "infinity"): one coalesced load of 32 row ends.
__device__ __forceinline__ int64_t row_end(const int32_t *rowptr, int M, int rb, int lane) {
    const int r = rb + 1 + lane;
    return r <= M ? (int64_t)__ldg(rowptr + r) : INT64_MAX;
}

// The row of each lane's entry e, given that every lane's entry lies in row rc or later and
// `end` holds row_end(rc) (loaded ahead by the caller).
__device__ __forceinline__ int rows_of_chunk(const int32_t *rowptr, int M, int rc, int64_t end, int64_t e,
                                             int lane) {
    int row = -1;
    for (int rb = rc;; rb += 32) {
        if (rb != rc) end = row_end(rowptr, M, rb, lane);  // a run of more than 32 row ends
        int lo = 0, len = 32;  // first k with end_k > e
#pragma unroll
        for (int it = 0; it < 6; ++it) {
            const int half = len >> 1;
            const int mid = lo + half;
            const int64_t v = __shfl_sync(FULL, end, mid < 32 ? mid : 31);
            const bool go = len > 0 && v <= e;
            lo = go ? mid + 1 : lo;
            len = len == 0 ? 0 : (go ? len - half - 1 : half);
        }
        if (row < 0 && lo < 32) row = rb + lo;
        if (__all_sync(FULL, row >= 0)) return row;
    }
}

// Entries [e0, e1), the first of which lies in row rc.  Per chunk: the column indices,
// values and 32 row ends of the next chunk are loaded while this one computes; the Y rows
// of U steps are gathered before any is used; a group fetches X_i only when its entry's
// row differs from the one it holds.
template <class EL, int LPN, int VPL, bool CHECK_COLS>
__device__ __forceinline__ void sddmm_entries(const SddmmProblem &P, int64_t e0, int64_t e1, int rc, int lane) {
    constexpr int U = LPN * VPL <= 8 ? LPN : (8 / VPL < 1 ? 1 : 8 / VPL);
    const int sl = lane % LPN, g = lane / LPN;
    using ST = typename EL::stored;
    const ST *X = static_cast<const ST *>(P.X);
    const uint4 *Yv = static_cast<const uint4 *>(P.Y) + sl;
    const int64_t ldv = P.ldy / EL::V;
    bool colok[VPL];
    int k0[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        k0[v] = (v * LPN + sl) * EL::V;
        colok[v] = !CHECK_COLS || k0[v] < P.Kd;
    }
    float x[VPL][EL::V];
    int xrow = -1;

    int c = 0;
    float s = 0.f;
    if (e0 + lane < e1) {
        c = ld_stream(P.colidx + e0 + lane);
        s = ld_stream(P.svals + e0 + lane);
    }
    int64_t end = row_end(P.rowptr, P.M, rc, lane);
    for (int64_t base = e0; base < e1; base += 32) {
        const int64_t nb = base + 32;
        int c2 = 0;
        float s2 = 0.f;
        if (nb + lane < e1) {
            c2 = ld_stream(P.colidx + nb + lane);
            s2 = ld_stream(P.svals + nb + lane);
        }
        const int cnt = e1 - base < 32 ? (int)(e1 - base) : 32;
        const int row = rows_of_chunk(P.rowptr, P.M, rc, end, lane < cnt ? base + lane : base, lane);
        rc = __shfl_sync(FULL, row, cnt - 1);
        if (nb < e1) end = row_end(P.rowptr, P.M, rc, lane);  // for the next chunk
        float part[LPN];
#pragma unroll
        for (int t0 = 0; t0 < LPN; t0 += U) {
            uint4 ry[U][VPL];
            int rr[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = g * LPN + t0 + u;
                const int cj = __shfl_sync(FULL, c, idx);
                rr[u] = __shfl_sync(FULL, row, idx);
                const uint4 *rp = Yv + (int64_t)cj * ldv;
#pragma unroll
                for (int v = 0; v < VPL; ++v)
                    ry[u][v] = idx < cnt && colok[v] ? ld_gather16(rp + v * LPN) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (rr[u] != xrow) {  // this group's entry starts another row: fetch its X row
                    xrow = rr[u];
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        uint4 raw = make_uint4(0, 0, 0, 0);
                        if (colok[v]) raw = ld_gather16(X + (int64_t)xrow * P.ldx + k0[v]);
                        EL::unpack(raw, x[v]);
                    }
                }
                float2 sum = make_float2(0.f, 0.f);
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    float y[EL::V];
                    EL::unpack(ry[u][v], y);
                    dot2(x[v], y, sum);
                }
                part[t0 + u] = sum.x + sum.y;
            }
        }
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
        if (lane < cnt) {
            float r = s * part[0];
            if (EL::dtype == GBSP_E4M3) r *= __ldg(P.x_scale + row) * __ldg(P.y_scale + c);
            __stcs(P.out + base + lane, r);
        }
        c = c2;
        s = s2;
    }
}

// Stored entries split evenly across the nwarps warps of the grid, in whole chunks of 32
// (nnz is read on the device, so the launch needs no host-side statistics).
template <class EL, int LPN, int VPL>
__global__ void __launch_bounds__(256) sddmm_entry_kernel(const SddmmProblem P, int nwarps) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t rnnz = __ldg(P.rowptr + P.M);
    const int64_t nnz = P.nnz >= 0 && P.nnz < rnnz ? P.nnz : rnnz;
    const int64_t chunks_per_warp = ((nnz + 31) / 32 + nwarps - 1) / nwarps;
    const int64_t e0 = min(w * chunks_per_warp * 32, nnz);
    const int64_t e1 = min(e0 + chunks_per_warp * 32, nnz);
    if (e0 >= e1) return;
    const int rc = row_of_entry(P.rowptr, P.M, e0, lane);
    if (P.Kd == LPN * VPL * EL::V)
        sddmm_entries<EL, LPN, VPL, false>(P, e0, e1, rc, lane);
    else
        sddmm_entries<EL, LPN, VPL, true>(P, e0, e1, rc, lane);
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

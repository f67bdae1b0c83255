// SpMM kernels (Eq. 1): C[i, :] = sum over the stored entries p of row i of a_p * B[colidx[p], :].
//
// Lane layout shared by every vectorised kernel: a warp splits into G = 32 / LPN groups
// of LPN lanes.  One group takes one nonzero at a time; each of its lanes gathers VPL
// 16-byte vectors (EL::V elements each) of the B row colidx[p], so a group covers
// LPN * VPL * EL::V columns of one column tile.  U gathers are issued per lane before
// any of them is consumed, so a warp keeps U * G row loads in flight.  Column indices and
// coefficients are read 32 at a time with one coalesced load per lane and handed to the
// groups by warp shuffles; the next 32 are prefetched while the current ones are used.
#pragma once

#include "common.cuh"

namespace gbsp {
namespace spmm_detail {

// Coefficient of stored entry p: the A value as FP32; for E4M3 it also folds in the
// per-row scale t_k of the gathered B row (the row scale s_i of A is applied at the end).
template <class EL>
__device__ __forceinline__ float coef(const SpmmProblem &P, int64_t p, int c) {
    const typename EL::stored *vals = static_cast<const typename EL::stored *>(P.vals);
    float a = EL::value(ld_stream(vals + p));
    if (EL::dtype == GBSP_E4M3) a *= __ldg(P.b_scale + c);
    return a;
}

// Where a lane's vectors sit in its group's column tile: vector v * LPN + sl (each load
// instruction of a group reads one contiguous span), or, paired (VPL = 2), 2 * sl + v, the
// two adjacent vectors arriving by one 32-byte load.
template <int LPN, bool PAIR>
__device__ __forceinline__ int lane_vec(int sl, int v) {
    return PAIR ? 2 * sl + v : v * LPN + sl;
}

// One step of a group: U nonzeros per group (G * U per warp), VPL 16-byte vectors per lane
// each.  CHECK_NNZ guards a partial chunk (entries past cnt are skipped), CHECK_COLS a
// partial column tile (vectors past N are skipped); the full-chunk, full-tile case issues
// its loads unpredicated.  Bv points at the lane's first vector (lane_vec(sl, 0)).
template <class EL, int LPN, int VPL, int U, bool CHECK_COLS, bool CHECK_NNZ, bool PAIR = false>
__device__ __forceinline__ void gather_step(const uint4 *__restrict__ Bv, int64_t ldv, int c, float a, int q,
                                            int cnt, int sub, const bool (&colok)[VPL],
                                            float (&acc)[VPL][EL::V]) {
    constexpr int G = 32 / LPN;
    static_assert(!PAIR || VPL == 2, "pairs are two vectors");
    uint4 raw[U][VPL];
    float aj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = q + u * G + sub;
        const int cj = __shfl_sync(FULL, c, idx);
        aj[u] = __shfl_sync(FULL, a, idx);
        const uint4 *rp = Bv + (int64_t)cj * ldv;
        if constexpr (PAIR) {
            bool ok = true, ok1 = true;
            if constexpr (CHECK_NNZ) ok = idx < cnt;
            if constexpr (CHECK_COLS) {
                ok1 = ok && colok[VPL - 1];
                ok = ok && colok[0];
            }
            if (ok1) {
                ld_gather32(rp, raw[u][0], raw[u][VPL - 1]);
            } else {  // the tile's last pair is cut by N (or the entry is past the chunk)
                raw[u][0] = ok ? ld_gather16(rp) : make_uint4(0, 0, 0, 0);
                raw[u][VPL - 1] = make_uint4(0, 0, 0, 0);
            }
            continue;
        }
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            if constexpr (CHECK_COLS || CHECK_NNZ) {
                bool ok = true;
                if constexpr (CHECK_NNZ) ok = idx < cnt;
                if constexpr (CHECK_COLS) ok = ok && colok[v];
                raw[u][v] = ok ? ld_gather16(rp + v * LPN) : make_uint4(0, 0, 0, 0);
            } else {
                raw[u][v] = ld_gather16(rp + v * LPN);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) EL::axpy(aj[u], raw[u][v], acc[v]);
    }
}

// Accumulates the stored entries [p0, p1) of one row into acc (the lane's VPL vectors of
// the row's column tile starting at col_base).
template <class EL, int LPN, int VPL, int U, bool CHECK_COLS, bool PAIR = false>
__device__ __forceinline__ void gather_range(const SpmmProblem &P, int64_t p0, int64_t p1,
                                             float (&acc)[VPL][EL::V], int lane, int col_base) {
    constexpr int G = 32 / LPN;
    constexpr int STEP = G * U;
    static_assert(STEP <= 32 && 32 % STEP == 0, "a chunk of 32 nonzeros must hold whole steps");
    const int sub = lane / LPN;
    const uint4 *Bv = static_cast<const uint4 *>(P.B) + col_base / EL::V;
    const int64_t ldv = P.ldb / EL::V;
    bool colok[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
        colok[v] = col_base + (lane_vec<LPN, PAIR>(0, v) - lane_vec<LPN, PAIR>(0, 0)) * EL::V < P.N;

    int c = 0;
    float a = 0.f;
    int64_t base = p0;
    if (base + lane < p1) {
        c = ld_stream(P.colidx + base + lane);
        a = coef<EL>(P, base + lane, c);
    }
    while (base < p1) {
        const int64_t nb = base + 32;
        int c2 = 0;
        float a2 = 0.f;
        if (nb + lane < p1) {
            c2 = ld_stream(P.colidx + nb + lane);
            a2 = coef<EL>(P, nb + lane, c2);
        }
        if (nb <= p1) {
#pragma unroll
            for (int q = 0; q < 32; q += STEP)
                gather_step<EL, LPN, VPL, U, CHECK_COLS, false, PAIR>(Bv, ldv, c, a, q, 32, sub, colok, acc);
        } else {
            // the row's last, partial chunk: whole steps unchecked, then the rest (fewer than
            // STEP entries) in predicated steps of UT = U / 2 slots per lane, whose gathers
            // are in flight together (one round trip per step rather than per entry) while a
            // short tail wastes at most half of a step's slots
            constexpr int UT = U > 1 ? U / 2 : 1;
            const int cnt = (int)(p1 - base);
            int q = 0;
#pragma unroll 1
            for (; q + STEP <= cnt; q += STEP)
                gather_step<EL, LPN, VPL, U, CHECK_COLS, false, PAIR>(Bv, ldv, c, a, q, cnt, sub, colok, acc);
#pragma unroll 1
            for (; q < cnt; q += G * UT)
                gather_step<EL, LPN, VPL, UT, CHECK_COLS, true, PAIR>(Bv, ldv, c, a, q, cnt, sub, colok, acc);
        }
        base = nb;
        c = c2;
        a = a2;
    }
}

// Sums the G group partials (xor butterfly across groups) so every group holds the row.
template <class EL, int LPN, int VPL>
__device__ __forceinline__ void reduce_groups(float (&acc)[VPL][EL::V]) {
#pragma unroll
    for (int off = LPN; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int k = 0; k < EL::V; ++k) acc[v][k] += __shfl_xor_sync(FULL, acc[v][k], off);
}

template <class EL, int LPN, int VPL, bool PAIR = false>
__device__ __forceinline__ void store_row(float *dst_row, const float (&acc)[VPL][EL::V], int lane,
                                          int col_base, int N, float scale) {
    if (lane >= LPN) return;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int col = col_base + (lane_vec<LPN, PAIR>(0, v) - lane_vec<LPN, PAIR>(0, 0)) * EL::V;
        if (col < N) {
#pragma unroll
            for (int k = 0; k < EL::V; k += 4)
                __stcs(reinterpret_cast<float4 *>(dst_row + col + k),
                       make_float4(acc[v][k] * scale, acc[v][k + 1] * scale, acc[v][k + 2] * scale,
                                   acc[v][k + 3] * scale));
        }
    }
}

template <class EL>
__device__ __forceinline__ float row_scale(const SpmmProblem &P, int row) {
    return EL::dtype == GBSP_E4M3 ? __ldg(P.a_scale + row) : 1.0f;
}

// One warp per row; blockIdx.y is the column tile.  PAIR: 32-byte aligned B rows (the
// launcher checks).
template <class EL, int LPN, int VPL, int U, bool PAIR = false>
__global__ void __launch_bounds__(256) spmm_rowsplit_kernel(const SpmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int col_base = blockIdx.y * (LPN * VPL * EL::V) + lane_vec<LPN, PAIR>(lane % LPN, 0) * EL::V;
    float acc[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    if ((blockIdx.y + 1) * (LPN * VPL * EL::V) <= P.N)
        gather_range<EL, LPN, VPL, U, false, PAIR>(P, p0, p1, acc, lane, col_base);
    else
        gather_range<EL, LPN, VPL, U, true, PAIR>(P, p0, p1, acc, lane, col_base);
    reduce_groups<EL, LPN, VPL>(acc);
    store_row<EL, LPN, VPL, PAIR>(P.C + (int64_t)row * P.ldc, acc, lane, col_base, P.N, row_scale<EL>(P, row));
}

// nnz-balanced split: warp w takes the items [w * ipw, (w + 1) * ipw) of the merge path
// (M row ends + nnz entries).  Rows that end inside the range are written directly; the
// partial sum of the row still open at the range end goes to the carry arrays and is
// added by spmm_merge_fixup_kernel.  The grid is fixed on the host, nnz is read on the
// device, so the launch needs no host-side knowledge of the matrix.
template <class EL, int LPN, int VPL, int U, bool PAIR = false>
__global__ void __launch_bounds__(256) spmm_merge_kernel(const SpmmProblem P, int32_t *carry_row,
                                                         float *carry_val, int nwarps) {
    constexpr int TW = LPN * VPL * EL::V;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int col_base = blockIdx.y * TW + lane_vec<LPN, PAIR>(lane % LPN, 0) * EL::V;
    const int64_t nnz = __ldg(P.rowptr + P.M);
    const int64_t total = (int64_t)P.M + nnz;
    const int64_t ipw = (total + nwarps - 1) / nwarps;
    const int64_t d0 = min((int64_t)w * ipw, total);
    const int64_t d1 = min(d0 + ipw, total);
    const int x0 = merge_search(P.rowptr, P.M, nnz, d0, lane);
    const int x1 = merge_search(P.rowptr, P.M, nnz, d1, lane);
    int64_t p = d0 - x0;
    const int64_t y1 = d1 - x1;
    float acc[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
    const bool full_tile = (blockIdx.y + 1) * TW <= P.N;
    for (int row = x0; row < x1; ++row) {
        const int64_t e = __ldg(P.rowptr + row + 1);
        if (full_tile)
            gather_range<EL, LPN, VPL, U, false, PAIR>(P, p, e, acc, lane, col_base);
        else
            gather_range<EL, LPN, VPL, U, true, PAIR>(P, p, e, acc, lane, col_base);
        reduce_groups<EL, LPN, VPL>(acc);
        store_row<EL, LPN, VPL, PAIR>(P.C + (int64_t)row * P.ldc, acc, lane, col_base, P.N, row_scale<EL>(P, row));
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
        p = e;
    }
    if (full_tile)
        gather_range<EL, LPN, VPL, U, false, PAIR>(P, p, y1, acc, lane, col_base);
    else
        gather_range<EL, LPN, VPL, U, true, PAIR>(P, p, y1, acc, lane, col_base);
    reduce_groups<EL, LPN, VPL>(acc);
    float *cv = carry_val + ((int64_t)blockIdx.y * nwarps + w) * TW;
    if (lane < LPN) {
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int k = 0; k < EL::V; k += 4)
                *reinterpret_cast<float4 *>(cv + lane_vec<LPN, PAIR>(lane, v) * EL::V + k) =
                    make_float4(acc[v][k], acc[v][k + 1], acc[v][k + 2], acc[v][k + 3]);
    }
    if (lane == 0 && blockIdx.y == 0) carry_row[w] = (d0 < d1 && x1 < P.M) ? x1 : -1;
}

// Adds the carries: the first warp of each run of equal carry rows sums the run in warp
// order (deterministic) and adds it, times the row scale, into C.
template <class EL>
__global__ void __launch_bounds__(256) spmm_merge_fixup_kernel(const SpmmProblem P, const int32_t *carry_row,
                                                               const float *carry_val, int nwarps, int TW) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nwarps) return;
    const int r = carry_row[w];
    if (r < 0 || (w > 0 && carry_row[w - 1] == r)) return;
    const float sc = row_scale<EL>(P, r);
    for (int col = lane; col < TW; col += 32) {
        const int gcol = blockIdx.y * TW + col;
        if (gcol >= P.N) break;
        float s = 0.f;
        for (int w2 = w; w2 < nwarps && carry_row[w2] == r; ++w2)
            s += carry_val[((int64_t)blockIdx.y * nwarps + w2) * TW + col];
        float *dst = P.C + (int64_t)r * P.ldc + gcol;
        *dst += s * sc;
    }
}

// Several consecutive rows per warp, one lane group of LPN lanes each (G = 32 / LPN rows
// per warp): the plan-free form of the hyper-sparse treatment, for matrices whose rows hold
// a few entries, where one warp per row leaves most of its groups idle.  Every lane of a
// group gathers its VPL vectors of each entry's B row, U entries in flight; the group's
// lanes load the same index and value (one broadcast) and no cross-group reduction is
// needed.  A long row keeps its group busy alone, so this layout only suits short rows.
template <class EL, int LPN, int VPL, int U>
__global__ void __launch_bounds__(256) spmm_rowgroup_kernel(const SpmmProblem P) {
    constexpr int G = 32 / LPN;
    constexpr int TW = LPN * VPL * EL::V;
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * G + lane / LPN;
    if (row >= P.M) return;  // a group's lanes share the row; no warp-wide exchange follows
    const int col_base = blockIdx.y * TW + (lane % LPN) * EL::V;
    const uint4 *Bv = static_cast<const uint4 *>(P.B) + col_base / EL::V;
    const int64_t ldv = P.ldb / EL::V;
    bool colok[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) colok[v] = col_base + v * LPN * EL::V < P.N;
    float acc[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    for (int64_t p = p0; p < p1; p += U) {
        int c[U];
        float a[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = p + u < p1;
            c[u] = ok[u] ? ld_stream(P.colidx + p + u) : 0;
            a[u] = ok[u] ? coef<EL>(P, p + u, c[u]) : 0.f;
        }
        uint4 raw[U][VPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                raw[u][v] = (ok[u] && colok[v]) ? ld_gather16(Bv + (int64_t)c[u] * ldv + v * LPN)
                                                : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < VPL; ++v) EL::axpy(a[u], raw[u][v], acc[v]);
    }
    const float sc = row_scale<EL>(P, (int)row);
    float *dst = P.C + row * P.ldc;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int col = col_base + v * LPN * EL::V;
        if (col < P.N) {
#pragma unroll
            for (int k = 0; k < EL::V; k += 4)
                __stcs(reinterpret_cast<float4 *>(dst + col + k),
                       make_float4(acc[v][k] * sc, acc[v][k + 1] * sc, acc[v][k + 2] * sc, acc[v][k + 3] * sc));
        }
    }
}

// Unvectorised form for any width and alignment: one warp per row, lane l owns columns
// l, l + 32, l + 64, l + 96 of a 128-column pass.
template <class EL>
__global__ void __launch_bounds__(256) spmm_scalar_kernel(const SpmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    const typename EL::stored *B = static_cast<const typename EL::stored *>(P.B);
    const float sc = row_scale<EL>(P, row);
    for (int c0 = blockIdx.y * 128; c0 < P.N; c0 += gridDim.y * 128) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t base = p0; base < p1; base += 32) {
            int c = 0;
            float a = 0.f;
            if (base + lane < p1) {
                c = ld_stream(P.colidx + base + lane);
                a = coef<EL>(P, base + lane, c);
            }
            const int cnt = (int)min((int64_t)32, p1 - base);
            for (int j = 0; j < cnt; ++j) {
                const int cj = __shfl_sync(FULL, c, j);
                const float aj = __shfl_sync(FULL, a, j);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int col = c0 + lane + 32 * t;
                    if (col < P.N) acc[t] = fmaf(aj, EL::scalar(B + (int64_t)cj * P.ldb + col), acc[t]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int col = c0 + lane + 32 * t;
            if (col < P.N) P.C[(int64_t)row * P.ldc + col] = acc[t] * sc;
        }
    }
}

}  // namespace spmm_detail

}  // namespace gbsp

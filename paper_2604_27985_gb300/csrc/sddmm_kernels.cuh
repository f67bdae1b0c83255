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

template <class EL, int LPN, int VPL>
__global__ void __launch_bounds__(256) sddmm_rowsplit_kernel(const SddmmProblem P) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= P.M) return;
    const int sl = lane % LPN, g = lane / LPN;
    using ST = typename EL::stored;
    const ST *X = static_cast<const ST *>(P.X);
    const ST *Y = static_cast<const ST *>(P.Y);

    bool colok[VPL];
    float x[VPL][EL::V];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int k0 = (v * LPN + sl) * EL::V;
        colok[v] = k0 < P.Kd;
        uint4 raw = make_uint4(0, 0, 0, 0);
        if (colok[v]) raw = ld_gather16(X + (int64_t)row * P.ldx + k0);
        EL::unpack(raw, x[v]);
    }
    const float xs = EL::dtype == GBSP_E4M3 ? __ldg(P.x_scale + row) : 1.0f;

    const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
    for (int64_t base = p0; base < p1; base += 32) {
        const bool mine = base + lane < p1;
        int c = 0;
        float s = 0.f;
        if (mine) {
            c = ld_stream(P.colidx + base + lane);
            s = ld_stream(P.svals + base + lane);
        }
        const int cnt = (int)min((int64_t)32, p1 - base);
        float part[LPN];
#pragma unroll
        for (int t = 0; t < LPN; ++t) {
            const int idx = g * LPN + t;
            const int cj = __shfl_sync(FULL, c, idx);
            const bool ok = idx < cnt;
            float sum = 0.f;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                uint4 raw = make_uint4(0, 0, 0, 0);
                if (ok && colok[v]) raw = ld_gather16(Y + (int64_t)cj * P.ldy + (v * LPN + sl) * EL::V);
                float y[EL::V];
                EL::unpack(raw, y);
#pragma unroll
                for (int k = 0; k < EL::V; ++k) sum = fmaf(x[v][k], y[k], sum);
            }
            part[t] = sum;
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
        if (mine) {
            float r = s * part[0];
            if (EL::dtype == GBSP_E4M3) r *= xs * __ldg(P.y_scale + c);
            __stcs(P.out + base + lane, r);
        }
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

// Host-side choice of lane layout and launch shape for the SpMM kernels: one translation
// unit per (element type, algorithm) instantiates launch_spmm_algo.
#pragma once

#include "spmm_kernels.cuh"

namespace gbsp {
namespace spmm_detail {

template <class EL, int LPN, int VPL, int U, int ALGO, bool PAIR = false>
int run(const SpmmProblem &P, int ctas_per_sm, cudaStream_t s) {
    constexpr int TW = LPN * VPL * EL::V;
    const int ntiles = (P.N + TW - 1) / TW;
    if constexpr (ALGO == GBSP_VARIANT_MERGE) {
        int per_sm = ctas_per_sm;
        if (per_sm <= 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmm_merge_kernel<EL, LPN, VPL, U, PAIR>, 256,
                                                              0) != cudaSuccess)
                return check_launch("occupancy query");
            per_sm = per_sm < 1 ? 1 : per_sm;
        }
        const int nblocks = sm_count() * per_sm;
        const int nwarps = nblocks * 8;
        void *cr = nullptr, *cv = nullptr;
        int st = scratch_alloc(&cr, sizeof(int32_t) * (size_t)nwarps, s);
        if (st != GBSP_OK) return st;
        st = scratch_alloc(&cv, sizeof(float) * (size_t)nwarps * ntiles * TW, s);
        if (st != GBSP_OK) {
            scratch_free(cr, s);
            return st;
        }
        spmm_merge_kernel<EL, LPN, VPL, U, PAIR><<<dim3(nblocks, ntiles), 256, 0, s>>>(
            P, static_cast<int32_t *>(cr), static_cast<float *>(cv), nwarps);
        spmm_merge_fixup_kernel<EL><<<dim3((nwarps + 7) / 8, ntiles), 256, 0, s>>>(
            P, static_cast<const int32_t *>(cr), static_cast<const float *>(cv), nwarps, TW);
        count_launches(2);
        st = check_launch("spmm merge");
        scratch_free(cv, s);
        scratch_free(cr, s);
        return st;
    } else if constexpr (ALGO == GBSP_VARIANT_ROWGROUP) {
        constexpr int G = 32 / LPN;
        const int64_t blocks = ((int64_t)P.M + 8 * G - 1) / (8 * G);
        spmm_rowgroup_kernel<EL, LPN, VPL, U><<<dim3((unsigned)blocks, ntiles), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("spmm rowgroup");
    } else {
        spmm_rowsplit_kernel<EL, LPN, VPL, U, PAIR><<<dim3((P.M + 7) / 8, ntiles), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("spmm rowsplit");
    }
}

// Gathers in flight per lane: U <= LPN keeps a step inside one chunk of 32 nonzeros,
// VPL * U <= 16 bounds the registers holding loads in flight.
template <class EL, int LPN, int VPL, int ALGO, bool PAIR = false>
int by_unroll(const SpmmProblem &P, int u, int cps, cudaStream_t s) {
    constexpr int UMAX = LPN < 16 / VPL ? LPN : 16 / VPL;
    if constexpr (UMAX >= 8) {
        if (u >= 8) return run<EL, LPN, VPL, 8, ALGO, PAIR>(P, cps, s);
    }
    if constexpr (UMAX >= 4) {
        if (u >= 4) return run<EL, LPN, VPL, 4, ALGO, PAIR>(P, cps, s);
    }
    if constexpr (UMAX >= 2) {
        return run<EL, LPN, VPL, 2, ALGO, PAIR>(P, cps, s);
    } else {
        return run<EL, LPN, VPL, 1, ALGO, PAIR>(P, cps, s);
    }
}

template <class EL, int VPL, int ALGO, bool PAIR = false>
int by_lanes(const SpmmProblem &P, int lpn, int u, int cps, cudaStream_t s) {
    if constexpr (VPL * EL::V > 16) {  // at most 16 accumulators per lane
        return fail(GBSP_ERR_UNSUPPORTED, "spmm: %d vectors per lane exceed 16 elements", VPL);
    } else switch (lpn) {
        case 1: if constexpr (VPL == 1) return by_unroll<EL, 1, 1, ALGO>(P, u, cps, s); break;
        case 2: if constexpr (VPL == 1) return by_unroll<EL, 2, 1, ALGO>(P, u, cps, s); break;
        case 4: if constexpr (VPL <= 2) return by_unroll<EL, 4, VPL, ALGO, PAIR>(P, u, cps, s); break;
        case 8: return by_unroll<EL, 8, VPL, ALGO, PAIR>(P, u, cps, s);
        case 16: return by_unroll<EL, 16, VPL, ALGO, PAIR>(P, u, cps, s);
        case 32: return by_unroll<EL, 32, VPL, ALGO, PAIR>(P, u, cps, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "spmm: no kernel for %d lanes x %d vectors", lpn, VPL);
}

}  // namespace spmm_detail

// Lane layout: VPL vectors per lane (default 2 once a row spans 16 vectors, else 1, so a
// row keeps at least 8 lanes and every load instruction covers whole 128-byte lines; at
// most 16 / V so a lane holds at most 16 accumulators) and LPN = the power of two covering
// the row's vectors, at most 32 (wider rows take several column tiles).  Layouts with
// VPL > 1 need at least 4 (VPL = 2) or 8 (VPL = 4) lanes.
inline void spmm_layout(int nvec, int vecs, int max_vpl, int &lpn, int &vpl) {
    vpl = vecs > 0 ? vecs : (nvec >= 16 ? 2 : 1);
    if (vpl > max_vpl) vpl = max_vpl;
    lpn = next_pow2((nvec + vpl - 1) / vpl);
    if (lpn > 32) lpn = 32;
    while ((vpl == 4 && lpn < 8) || (vpl == 2 && lpn < 4)) {
        vpl >>= 1;
        lpn = next_pow2((nvec + vpl - 1) / vpl);
        if (lpn > 32) lpn = 32;
    }
}

template <class EL, int ALGO>
int launch_spmm_algo(const SpmmProblem &P, int vecs, int unroll, int ctas_per_sm, cudaStream_t s) {
    using namespace spmm_detail;
    int lpn, vpl;
    spmm_layout(P.N / EL::V, vecs, 16 / EL::V, lpn, vpl);  // N % V == 0 is checked by the caller
    // Default layout for 128-byte rows (FP32 N = 32, BF16 N = 64) with 32-byte aligned B rows
    // (row split and merge path): 4 lanes per entry, each lane's two adjacent vectors by one
    // 32-byte load, 8 entries per step, instead of 8 lanes x one vector.  Measured on 65,536^2
    // at 99%, BF16 N = 64: 0.335 against 0.393 ms.  Wider rows keep the strided layout, which
    // measured as fast (FP32 N = 64) or faster (BF16 N = 256: 0.61 against 0.67 ms paired);
    // explicit vecs keep it too.
    if constexpr (ALGO != GBSP_VARIANT_ROWGROUP && 2 * EL::V <= 16) {
        if (vecs == 0 && P.N / EL::V == 8 && aligned32(P.B) && P.ldb % (2 * EL::V) == 0)
            return by_lanes<EL, 2, ALGO, true>(P, 4, unroll > 0 ? unroll : 4, ctas_per_sm, s);
    }
    const int u = unroll > 0 ? unroll : (vpl == 1 ? 8 : 4);
    switch (vpl) {
        case 1: return by_lanes<EL, 1, ALGO>(P, lpn, u, ctas_per_sm, s);
        case 2: return by_lanes<EL, 2, ALGO>(P, lpn, u, ctas_per_sm, s);
        case 4: return by_lanes<EL, 4, ALGO>(P, lpn, u, ctas_per_sm, s);
    }
    return fail(GBSP_ERR_INVALID_ARG, "spmm: vectors per lane must be 1, 2 or 4");
}

}  // namespace gbsp

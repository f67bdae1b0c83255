// Host-side choice of lane layout and launch shape for the SpMM kernels of one element type.
#pragma once

#include "spmm_kernels.cuh"

namespace gbsp {
namespace spmm_detail {

template <class EL, int LPN, int VPL, int U>
int run(const SpmmProblem &P, int variant, int ctas_per_sm, cudaStream_t s) {
    constexpr int TW = LPN * VPL * EL::V;
    const int ntiles = (P.N + TW - 1) / TW;
    if (variant == GBSP_VARIANT_MERGE) {
        int per_sm = ctas_per_sm;
        if (per_sm <= 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmm_merge_kernel<EL, LPN, VPL, U>, 256, 0) !=
                cudaSuccess)
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
        spmm_merge_kernel<EL, LPN, VPL, U><<<dim3(nblocks, ntiles), 256, 0, s>>>(
            P, static_cast<int32_t *>(cr), static_cast<float *>(cv), nwarps);
        spmm_merge_fixup_kernel<EL><<<dim3((nwarps + 7) / 8, ntiles), 256, 0, s>>>(
            P, static_cast<const int32_t *>(cr), static_cast<const float *>(cv), nwarps, TW);
        count_launches(2);
        st = check_launch("spmm merge");
        scratch_free(cv, s);
        scratch_free(cr, s);
        return st;
    }
    spmm_rowsplit_kernel<EL, LPN, VPL, U><<<dim3((P.M + 7) / 8, ntiles), 256, 0, s>>>(P);
    count_launches(1);
    return check_launch("spmm rowsplit");
}

template <class EL, int LPN, int VPL>
int by_unroll(const SpmmProblem &P, int variant, int u, int cps, cudaStream_t s) {
    if constexpr (LPN >= 8) {
        if (u >= 8) return run<EL, LPN, VPL, 8>(P, variant, cps, s);
    }
    if constexpr (LPN >= 4) {
        if (u >= 4) return run<EL, LPN, VPL, 4>(P, variant, cps, s);
    }
    if constexpr (LPN >= 2) {
        return run<EL, LPN, VPL, 2>(P, variant, cps, s);
    } else {
        return run<EL, LPN, VPL, 1>(P, variant, cps, s);
    }
}

}  // namespace spmm_detail

template <class EL>
int launch_spmm_typed(const SpmmProblem &P, int variant, int unroll, int ctas_per_sm, cudaStream_t s) {
    using namespace spmm_detail;
    if (variant == GBSP_VARIANT_SCALAR) {
        spmm_scalar_kernel<EL><<<dim3((P.M + 7) / 8, 1), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("spmm scalar");
    }
    const int nvec = P.N / EL::V;  // N % V == 0 is checked by the caller
    const int u = unroll > 0 ? unroll : 4;
    if (nvec > 32) return by_unroll<EL, 32, 2>(P, variant, u, ctas_per_sm, s);
    switch (next_pow2(nvec)) {
        case 1: return by_unroll<EL, 1, 1>(P, variant, u, ctas_per_sm, s);
        case 2: return by_unroll<EL, 2, 1>(P, variant, u, ctas_per_sm, s);
        case 4: return by_unroll<EL, 4, 1>(P, variant, u, ctas_per_sm, s);
        case 8: return by_unroll<EL, 8, 1>(P, variant, u, ctas_per_sm, s);
        case 16: return by_unroll<EL, 16, 1>(P, variant, u, ctas_per_sm, s);
        default: return by_unroll<EL, 32, 1>(P, variant, u, ctas_per_sm, s);
    }
}

}  // namespace gbsp

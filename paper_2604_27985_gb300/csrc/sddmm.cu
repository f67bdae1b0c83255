// SDDMM launches for every element type of X and Y.
#include "sddmm_kernels.cuh"

namespace gbsp {
namespace sddmm_detail {

template <class EL, int LPN, int VPL, bool PAIR = false>
int run(const SddmmProblem &P, int variant, cudaStream_t s) {
    if (variant == GBSP_VARIANT_ENTRY) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sddmm_entry_kernel<EL, LPN, VPL>, 256, 0) !=
            cudaSuccess)
            return check_launch("occupancy query");
        const int nblocks = sm_count() * (per_sm < 1 ? 1 : per_sm);
        sddmm_entry_kernel<EL, LPN, VPL><<<dim3(nblocks), 256, 0, s>>>(P, nblocks * 8);
        count_launches(1);
        return check_launch("sddmm entry split");
    }
    if (variant == GBSP_VARIANT_MERGE) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sddmm_merge_kernel<EL, LPN, VPL, PAIR>, 256, 0) !=
            cudaSuccess)
            return check_launch("occupancy query");
        const int nblocks = sm_count() * (per_sm < 1 ? 1 : per_sm);
        sddmm_merge_kernel<EL, LPN, VPL, PAIR><<<dim3(nblocks), 256, 0, s>>>(P, nblocks * 8);
        count_launches(1);
        return check_launch("sddmm merge");
    }
    if (P.pos)  // a plan's residual: values and outputs at the entries' original positions
        sddmm_rowsplit_kernel<EL, LPN, VPL, true, PAIR><<<dim3((P.M + 7) / 8), 256, 0, s>>>(P);
    else
        sddmm_rowsplit_kernel<EL, LPN, VPL, false, PAIR><<<dim3((P.M + 7) / 8), 256, 0, s>>>(P);
    count_launches(1);
    return check_launch("sddmm rowsplit");
}

template <class EL, int VPL>
int by_lanes(const SddmmProblem &P, int lpn, int variant, cudaStream_t s) {
    if constexpr (VPL * EL::V > 16) {  // at most 16 elements of X_i per lane
        return fail(GBSP_ERR_UNSUPPORTED, "sddmm: %d vectors per lane exceed 16 elements", VPL);
    } else switch (lpn) {
        case 1: if constexpr (VPL == 1) return run<EL, 1, 1>(P, variant, s); break;
        case 2: if constexpr (VPL == 1) return run<EL, 2, 1>(P, variant, s); break;
        case 4: if constexpr (VPL <= 2) return run<EL, 4, VPL>(P, variant, s); break;
        case 8: return run<EL, 8, VPL>(P, variant, s);
        case 16: return run<EL, 16, VPL>(P, variant, s);
        case 32: return run<EL, 32, VPL>(P, variant, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "sddmm: no kernel for %d lanes x %d vectors", lpn, VPL);
}

}  // namespace sddmm_detail

// Lane layout: VPL vectors per lane (default 2 from 8 vectors per row, 4 from 32; at most
// 16 / V; measured best on 65,536^2 at 99% for Kd = 32..256) and LPN lanes covering the
// row, at most 32.  Layouts with VPL > 1 need at least 4 (VPL = 2) or 8 (VPL = 4) lanes.
template <class EL>
int launch_sddmm_typed(const SddmmProblem &P, int variant, int vecs, cudaStream_t s) {
    using namespace sddmm_detail;
    if (variant == GBSP_VARIANT_SCALAR) {
        sddmm_scalar_kernel<EL><<<dim3((P.M + 7) / 8), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("sddmm scalar");
    }
    const int nvec = P.Kd / EL::V;
    const int max_vpl = 16 / EL::V;
    // Paired layout (FP32): each lane fetches two adjacent 16-byte vectors with one 32-byte
    // load, half the lanes per entry of the one-vector layout (so one reduce-scatter round
    // less and twice the entries per step) and half its load instructions.  Rows of 8 to 64
    // vectors, 32-byte aligned X and Y rows.  Measured on 65,536^2 at 99%, Kd = 32: 0.299
    // against 0.347 ms (4.5 against 6.6 warp instructions per entry); at 16,384^2, Kd = 256:
    // 1% to 9% faster.  BF16 measured slower paired (Kd = 32: 0.262 against 0.235 ms; Kd =
    // 256: 2-4%), where the mixed-precision dot already left fewer instructions per entry.
    const bool pairable = EL::dtype == GBSP_F32 && vecs == 0 && nvec >= 8 && nvec <= 64 && (nvec & (nvec - 1)) == 0 &&
                          aligned32(P.X) && aligned32(P.Y) && P.ldx % (2 * EL::V) == 0 && P.ldy % (2 * EL::V) == 0;
    if (pairable && variant != GBSP_VARIANT_ENTRY) {
        switch (nvec / 2) {
            case 4: return run<EL, 4, 2, true>(P, variant, s);
            case 8: return run<EL, 8, 2, true>(P, variant, s);
            case 16: return run<EL, 16, 2, true>(P, variant, s);
            case 32: return run<EL, 32, 2, true>(P, variant, s);
        }
    }
    // one vector per lane up to 8 vectors (8 lanes x 16 B read a 128-byte row in one
    // wavefront; measured 3% faster than 4 x 2 at Kd = 32 FP32), then 2 or 4
    int vpl = vecs > 0 ? vecs : (nvec >= 32 ? 4 : nvec > 8 ? 2 : 1);
    if (vpl > max_vpl) vpl = max_vpl;
    if (nvec > 32 * vpl) vpl = nvec > 64 ? 4 : 2;
    if (vpl > max_vpl)
        return fail(GBSP_ERR_UNSUPPORTED, "sddmm: Kd = %d is wider than 32 lanes x %d elements", P.Kd, 16);
    int lpn = next_pow2((nvec + vpl - 1) / vpl);
    while ((vpl == 4 && lpn < 8) || (vpl == 2 && lpn < 4)) {
        vpl >>= 1;
        lpn = next_pow2((nvec + vpl - 1) / vpl);
    }
    if (lpn > 32) return fail(GBSP_ERR_UNSUPPORTED, "sddmm: Kd = %d too wide for %d vectors per lane", P.Kd, vpl);
    switch (vpl) {
        case 1: return by_lanes<EL, 1>(P, lpn, variant, s);
        case 2: return by_lanes<EL, 2>(P, lpn, variant, s);
        case 4: return by_lanes<EL, 4>(P, lpn, variant, s);
    }
    return fail(GBSP_ERR_INVALID_ARG, "sddmm: vectors per lane must be 1, 2 or 4");
}

template int launch_sddmm_typed<F32>(const SddmmProblem &, int, int, cudaStream_t);
template int launch_sddmm_typed<BF16>(const SddmmProblem &, int, int, cudaStream_t);
template int launch_sddmm_typed<E4M3>(const SddmmProblem &, int, int, cudaStream_t);

}  // namespace gbsp

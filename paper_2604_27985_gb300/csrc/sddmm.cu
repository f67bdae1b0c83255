// SDDMM launches for every element type of X and Y.
#include "sddmm_kernels.cuh"

namespace gbsp {
namespace sddmm_detail {

template <class EL, int LPN, int VPL>
int run(const SddmmProblem &P, cudaStream_t s) {
    sddmm_rowsplit_kernel<EL, LPN, VPL><<<dim3((P.M + 7) / 8), 256, 0, s>>>(P);
    count_launches(1);
    return check_launch("sddmm rowsplit");
}

}  // namespace sddmm_detail

template <class EL>
int launch_sddmm_typed(const SddmmProblem &P, int variant, cudaStream_t s) {
    using namespace sddmm_detail;
    if (variant == GBSP_VARIANT_SCALAR) {
        sddmm_scalar_kernel<EL><<<dim3((P.M + 7) / 8), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("sddmm scalar");
    }
    const int nvec = P.Kd / EL::V;  // Kd % V == 0 and Kd <= 128 * V are checked by the caller
    if (nvec > 64) return run<EL, 32, 4>(P, s);
    if (nvec > 32) return run<EL, 32, 2>(P, s);
    switch (next_pow2(nvec)) {
        case 1: return run<EL, 1, 1>(P, s);
        case 2: return run<EL, 2, 1>(P, s);
        case 4: return run<EL, 4, 1>(P, s);
        case 8: return run<EL, 8, 1>(P, s);
        case 16: return run<EL, 16, 1>(P, s);
        default: return run<EL, 32, 1>(P, s);
    }
}

template int launch_sddmm_typed<F32>(const SddmmProblem &, int, cudaStream_t);
template int launch_sddmm_typed<BF16>(const SddmmProblem &, int, cudaStream_t);
template int launch_sddmm_typed<E4M3>(const SddmmProblem &, int, cudaStream_t);

}  // namespace gbsp

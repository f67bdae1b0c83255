// SpMM dispatch by element type and algorithm, and the unvectorised kernel.
#include "spmm_kernels.cuh"

namespace gbsp {

template <class EL>
int launch_spmm_typed(const SpmmProblem &P, int variant, int vecs, int unroll, int ctas_per_sm, cudaStream_t s) {
    if (variant == GBSP_VARIANT_SCALAR) {
        spmm_detail::spmm_scalar_kernel<EL><<<dim3((P.M + 7) / 8, 1), 256, 0, s>>>(P);
        count_launches(1);
        return check_launch("spmm scalar");
    }
    if (variant == GBSP_VARIANT_MERGE) return launch_spmm_algo<EL, GBSP_VARIANT_MERGE>(P, vecs, unroll, ctas_per_sm, s);
    if (variant == GBSP_VARIANT_ROWGROUP)
        return launch_spmm_algo<EL, GBSP_VARIANT_ROWGROUP>(P, vecs, unroll, ctas_per_sm, s);
    return launch_spmm_algo<EL, GBSP_VARIANT_ROWSPLIT>(P, vecs, unroll, ctas_per_sm, s);
}

int launch_spmm(const SpmmProblem &p, int variant, int vecs, int unroll, int ctas_per_sm, cudaStream_t s) {
    switch (p.dtype) {
        case GBSP_F32: return launch_spmm_typed<F32>(p, variant, vecs, unroll, ctas_per_sm, s);
        case GBSP_BF16: return launch_spmm_typed<BF16>(p, variant, vecs, unroll, ctas_per_sm, s);
        case GBSP_E4M3: return launch_spmm_typed<E4M3>(p, variant, vecs, unroll, ctas_per_sm, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "spmm: dtype %d", p.dtype);
}

}  // namespace gbsp

// SpMM instantiation: BF16 operands, row-group kernels.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_algo<BF16, GBSP_VARIANT_ROWGROUP>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

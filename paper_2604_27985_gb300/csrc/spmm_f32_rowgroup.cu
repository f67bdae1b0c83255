// SpMM instantiation: F32 operands, row-group kernels.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_algo<F32, GBSP_VARIANT_ROWGROUP>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

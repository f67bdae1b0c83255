// SpMM instantiation: E4M3 operands, rowsplit kernels.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_algo<E4M3, GBSP_VARIANT_ROWSPLIT>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

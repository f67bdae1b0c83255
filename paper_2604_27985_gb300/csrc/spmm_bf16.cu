// SpMM instantiation for BF16 operands.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_typed<BF16>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

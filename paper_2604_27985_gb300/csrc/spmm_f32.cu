// SpMM instantiation for F32 operands.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_typed<F32>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

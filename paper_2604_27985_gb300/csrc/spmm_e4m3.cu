// SpMM instantiation for E4M3 operands.
#include "spmm_launch.cuh"

namespace gbsp {
template int launch_spmm_typed<E4M3>(const SpmmProblem &, int, int, int, cudaStream_t);
}  // namespace gbsp

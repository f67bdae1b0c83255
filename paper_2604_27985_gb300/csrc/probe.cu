// Gather-bandwidth probe (a measurement utility; no counterpart in the paper).
//
// The SpMM and SDDMM kernels spend their time gathering whole dense rows selected by a
// column-index stream.  When the gathered operand fits in L2, HBM is not what binds them;
// this kernel measures the ceiling of that access pattern on its own: the same lane layout
// (LPN lanes per row, VPL 16-byte vectors per lane, U gathers in flight per lane), the same
// coalesced index loads handed to the lane groups by shuffles, and no arithmetic beyond an
// XOR that keeps every load live.  Run over the workload's own column indices, its rows x
// row bytes / time is the gather peak the sparse kernels are held against.
#include "common.cuh"

namespace gbsp {
namespace {

template <int LPN, int VPL, int U>
__global__ void __launch_bounds__(256) gather_probe_kernel(const uint4 *__restrict__ table, int64_t ldv,
                                                           const int32_t *__restrict__ idx, int64_t n,
                                                           uint32_t *__restrict__ sink) {
    constexpr int G = 32 / LPN;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPN, sl = lane % LPN;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint4 *base_row = table + sl;
    uint32_t acc = 0;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        // rows past n (the last chunk) gather row 0, which always exists
        const int c = base + lane < n ? ld_stream(idx + base + lane) : 0;
#pragma unroll
        for (int t = 0; t < 32 / G; t += U) {
            uint4 r[U][VPL];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = __shfl_sync(FULL, c, g * (32 / G) + t + u);
#pragma unroll
                for (int v = 0; v < VPL; ++v) r[u][v] = ld_gather16(base_row + (int64_t)j * ldv + v * LPN);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < VPL; ++v) acc ^= r[u][v].x ^ r[u][v].y ^ r[u][v].z ^ r[u][v].w;
        }
    }
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int LPN, int VPL>
int launch_probe(const void *table, int64_t ld_bytes, const int32_t *idx, int64_t n, uint32_t *sink, int blocks,
                 int unroll, cudaStream_t s) {
    const uint4 *t = static_cast<const uint4 *>(table);
    if (unroll >= 8 && LPN >= 8)
        gather_probe_kernel<LPN, VPL, (LPN >= 8 ? 8 : 1)><<<blocks, 256, 0, s>>>(t, ld_bytes / 16, idx, n, sink);
    else
        gather_probe_kernel<LPN, VPL, (LPN >= 4 ? 4 : 1)><<<blocks, 256, 0, s>>>(t, ld_bytes / 16, idx, n, sink);
    count_launches(1);
    return check_launch("gather probe");
}

}  // namespace
}  // namespace gbsp

using namespace gbsp;

GBSP_EXPORT int gbsp_gather_probe(const void *table, int64_t rows, int64_t row_bytes, int64_t ld_bytes,
                                  const int32_t *idx, int64_t n, uint32_t *sink, int32_t blocks, int32_t unroll,
                                  void *stream) {
    if (!table || !idx || !sink || rows <= 0 || n < 0 || blocks <= 0)
        return fail(GBSP_ERR_INVALID_ARG, "gather probe: bad argument");
    if (row_bytes != 128 && row_bytes != 256 && row_bytes != 512 && row_bytes != 1024)
        return fail(GBSP_ERR_UNSUPPORTED, "gather probe: row_bytes must be 128, 256, 512 or 1024");
    if (ld_bytes < row_bytes || ld_bytes % 16 || !aligned16(table))
        return fail(GBSP_ERR_ALIGN, "gather probe: the table must be 16-byte aligned with ld_bytes a multiple of 16");
    if (n == 0) return ok();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st;
    if (row_bytes == 128)
        st = launch_probe<8, 1>(table, ld_bytes, idx, n, sink, blocks, unroll, s);
    else if (row_bytes == 256)
        st = launch_probe<8, 2>(table, ld_bytes, idx, n, sink, blocks, unroll, s);
    else if (row_bytes == 512)
        st = launch_probe<16, 2>(table, ld_bytes, idx, n, sink, blocks, unroll, s);
    else
        st = launch_probe<32, 2>(table, ld_bytes, idx, n, sink, blocks, unroll, s);
    return st ? st : ok();
}

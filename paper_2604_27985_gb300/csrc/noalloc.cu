// FP32 SpMM through the merge-path kernels with the carry scratch in a fixed device array,
// for callers that must not allocate device memory during the call.
//
// Who needs it: a caller whose device memory is entirely handed out by another allocator
// (a framework's caching allocator that reserved nearly all of HBM, a fixed arena in a
// serving process) can see a driver allocation fail at call time, and a latency-bound
// loop cannot afford an allocation that may synchronise.  The general entry points take
// their merge-path carry buffers from a library-owned pool, which neither caller can
// accept; this one takes them from a file-scope device array instead.
#include <mutex>

#include "spmm_kernels.cuh"

namespace gbsp {
namespace {

// One int32 carry row per warp and TW floats of carry values per warp and column tile.
constexpr size_t kCarryRowSlots = 16384;
constexpr size_t kScratchBytes = size_t(4) << 20;  // 4 MiB, held by every GPU that loads the library
constexpr size_t kCarryRowBytes = kCarryRowSlots * sizeof(int32_t);
constexpr size_t kCarryValBytes = kScratchBytes - kCarryRowBytes;
constexpr int64_t kMaxN = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device
// and kept for the life of the process (a cudaDeviceReset makes it stale; the header says
// so).  The host-side name of the array is only a stand-in, never a device address.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(GBSP_ERR_CUDA, "spmm_csr_noalloc: no current device");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GBSP_ERR_CUDA, "spmm_csr_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GBSP_OK;
}

template <int LPN, int VPL, int U>
int run_noalloc(const SpmmProblem &P, unsigned char *scratch, cudaStream_t s) {
    using namespace spmm_detail;
    constexpr int TW = LPN * VPL * F32::V;
    const int ntiles = (P.N + TW - 1) / TW;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmm_merge_kernel<F32, LPN, VPL, U>, 256, 0) !=
        cudaSuccess)
        return check_launch("spmm_csr_noalloc occupancy query");
    per_sm = per_sm < 1 ? 1 : per_sm;
    int64_t nwarps = (int64_t)sm_count() * per_sm * 8;
    const int64_t fit_vals = (int64_t)(kCarryValBytes / (sizeof(float) * (size_t)ntiles * TW));
    if (nwarps > fit_vals) nwarps = fit_vals;
    if (nwarps > (int64_t)kCarryRowSlots) nwarps = kCarryRowSlots;
    nwarps -= nwarps % 8;  // whole CTAs of 8 warps
    if (nwarps < 8) return fail(GBSP_ERR_INVALID_ARG, "spmm_csr_noalloc: N = %d does not fit the scratch", P.N);
    int32_t *carry_row = reinterpret_cast<int32_t *>(scratch);
    float *carry_val = reinterpret_cast<float *>(scratch + kCarryRowBytes);
    spmm_merge_kernel<F32, LPN, VPL, U><<<dim3((unsigned)(nwarps / 8), ntiles), 256, 0, s>>>(P, carry_row, carry_val,
                                                                                          (int)nwarps);
    spmm_merge_fixup_kernel<F32><<<dim3((unsigned)(nwarps / 8), ntiles), 256, 0, s>>>(P, carry_row, carry_val,
                                                                                      (int)nwarps, TW);
    count_launches(2);
    return check_launch("spmm_csr_noalloc");
}

}  // namespace
}  // namespace gbsp

using namespace gbsp;

GBSP_EXPORT int spmm_csr_noalloc(const int32_t *rowptr, const int32_t *colidx, const float *vals, const float *B,
                                 float *C, int64_t M, int64_t K, int64_t N, void *stream) {
    if (M < 0 || K < 0 || N < 0 || M > 2147483647LL || K > 2147483647LL)
        return fail(GBSP_ERR_INVALID_ARG, "spmm_csr_noalloc: sizes out of range");
    if (N > kMaxN)
        return fail(GBSP_ERR_INVALID_ARG, "spmm_csr_noalloc: N = %lld exceeds the maximum %lld that the fixed "
                    "%zu-byte scratch holds", (long long)N, (long long)kMaxN, kScratchBytes);
    if (M == 0 || N == 0) return ok();
    if (!rowptr || !colidx || !vals || !B || !C) return fail(GBSP_ERR_INVALID_ARG, "spmm_csr_noalloc: null pointer");
    if (N % 4 || !aligned16(B) || !aligned16(C))
        return fail(GBSP_ERR_ALIGN, "spmm_csr_noalloc: N must be a multiple of 4 and B, C 16-byte aligned");
    void *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st) return st;
    SpmmProblem p{};
    p.M = (int32_t)M;
    p.K = (int32_t)K;
    p.N = (int32_t)N;
    p.nnz = -1;
    p.rowptr = rowptr;
    p.colidx = colidx;
    p.vals = vals;
    p.B = B;
    p.ldb = N;
    p.C = C;
    p.ldc = N;
    p.dtype = GBSP_F32;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    const int nvec = (int)(N / 4);
    if (nvec > 32) st = run_noalloc<32, 2, 4>(p, sc, s);
    else {
        switch (next_pow2(nvec)) {
            case 1: st = run_noalloc<1, 1, 1>(p, sc, s); break;
            case 2: st = run_noalloc<2, 1, 2>(p, sc, s); break;
            case 4: st = run_noalloc<4, 1, 4>(p, sc, s); break;
            case 8: st = run_noalloc<8, 1, 4>(p, sc, s); break;
            case 16: st = run_noalloc<16, 1, 4>(p, sc, s); break;
            default: st = run_noalloc<32, 1, 4>(p, sc, s); break;
        }
    }
    return st ? st : ok();
}

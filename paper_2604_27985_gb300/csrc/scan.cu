// Exclusive prefix sum of int32 counts on the device (used by the condensed-tile plan).
#include "common.cuh"

namespace gbsp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < (kScanThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, s, off);
            if (lane >= off) s += y;
        }
        warp_sums[lane] = s;  // inclusive sums of the warps
    }
    __syncthreads();
    total = warp_sums[kScanThreads / 32 - 1];
    const int64_t before = warp == 0 ? 0 : warp_sums[warp - 1];
    __syncthreads();
    return before + x - v;
}

// Per tile: sum of its counts.
__global__ void __launch_bounds__(kScanThreads) tile_sums_kernel(const int32_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int64_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the tile sums in place (exclusive), looping over them.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t *sums, int64_t ntiles, int32_t *out_total,
                                                                 int64_t n) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, ws, total);
        if (i < ntiles) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) out_total[n] = (int32_t)carry;
}

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const int32_t *in, int64_t n, const int64_t *sums,
                                                                 int32_t *out) {
    __shared__ int64_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t run = sums[blockIdx.x] + block_exclusive_scan(s, ws, total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = (int32_t)run;
        run += v[i];
    }
}

}  // namespace

// out[0..n] = exclusive prefix sums of in[0..n) with out[n] the total.  The caller
// guarantees the total fits in int32.  in and out may not alias.
int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    const int64_t ntiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    void *sums = nullptr;
    int st = scratch_alloc(&sums, sizeof(int64_t) * (size_t)ntiles, s);
    if (st) return st;
    int64_t *sm = static_cast<int64_t *>(sums);
    if (n > 0) {
        tile_sums_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, sm);
    } else {
        cudaMemsetAsync(sm, 0, sizeof(int64_t), s);
    }
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sm, n > 0 ? ntiles : 0, out, n);
    if (n > 0) tile_scan_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, sm, out);
    count_launches(n > 0 ? 3 : 1);
    st = check_launch("scan");
    scratch_free(sums, s);
    return st;
}

}  // namespace gbsp

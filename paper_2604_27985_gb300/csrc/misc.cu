// CSR validation and the BF16 / E4M3 conversion kernels.
#include "common.cuh"

namespace gbsp {
namespace {

// Counts violations of: rowptr[0] = 0, rowptr non-decreasing, rowptr[rows] = nnz,
// 0 <= colidx < cols.  Integer atomics only, so the count is exact.
__global__ void validate_kernel(const int32_t *rowptr, const int32_t *colidx, int64_t rows, int64_t cols,
                                int64_t nnz, unsigned long long *count) {
    unsigned long long bad = 0;
    const int64_t n = rows > nnz ? rows : nnz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < rows && rowptr[i + 1] < rowptr[i]) ++bad;
        if (i < nnz) {
            const int c = colidx[i];
            if (c < 0 || c >= cols) ++bad;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rowptr[0] != 0) ++bad;
        if ((int64_t)rowptr[rows] != nnz) ++bad;
    }
    for (int off = 16; off > 0; off >>= 1) bad += __shfl_xor_sync(FULL, bad, off);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

__global__ void quant_bf16_kernel(const float *__restrict__ x, uint16_t *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
        out[i] = *reinterpret_cast<uint16_t *>(&h);
    }
}

// One warp per row: the row maximum |x| by a warp reduction, s = max / 448 (FP32
// division, 1 for an all-zero row), then each entry is the saturating round-to-nearest-even
// E4M3 of the FP32 quotient x / s.
__global__ void quant_e4m3_rows_kernel(const float *__restrict__ x, const int32_t *__restrict__ rowptr, int64_t nrows,
                                       int64_t ncols, int64_t ld, uint8_t *__restrict__ q, float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= nrows) return;
    const int64_t b = rowptr ? (int64_t)rowptr[r] : r * ld;
    const int64_t e = rowptr ? (int64_t)rowptr[r + 1] : r * ld + ncols;
    float amax = 0.f;
    for (int64_t p = b + lane; p < e; p += 32) amax = fmaxf(amax, fabsf(x[p]));
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    const float s = amax == 0.f ? 1.0f : __fdiv_rn(amax, 448.0f);
    if (lane == 0) scale[r] = s;
    for (int64_t p = b + lane; p < e; p += 32)
        q[p] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(x[p], s), __NV_SATFINITE, __NV_E4M3);
}

}  // namespace

int launch_validate(const gbsp_csr &A, unsigned long long *d_count, cudaStream_t s) {
    if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s) != cudaSuccess) return check_launch("validate memset");
    const int64_t n = A.rows > A.nnz ? A.rows : A.nnz;
    int64_t blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 16L * sm_count()) blocks = 16L * sm_count();
    validate_kernel<<<(unsigned)blocks, 256, 0, s>>>(A.rowptr, A.colidx, A.rows, A.cols, A.nnz, d_count);
    count_launches(1);
    return check_launch("validate");
}

int launch_quant_bf16(const float *x, uint16_t *out, int64_t n, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 32L * sm_count()) blocks = 32L * sm_count();
    quant_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, out, n);
    count_launches(1);
    return check_launch("quantize bf16");
}

int launch_quant_e4m3_rows(const float *x, const int32_t *rowptr, int64_t nrows, int64_t ncols, int64_t ld,
                           uint8_t *q, float *scale, cudaStream_t s) {
    quant_e4m3_rows_kernel<<<(unsigned)((nrows + 7) / 8), 256, 0, s>>>(x, rowptr, nrows, ncols, ld, q, scale);
    count_launches(1);
    return check_launch("quantize e4m3");
}

}  // namespace gbsp

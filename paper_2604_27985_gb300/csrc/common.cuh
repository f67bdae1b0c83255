// Internal helpers shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "gbsp.h"

#define GBSP_EXPORT extern "C" __attribute__((visibility("default")))

namespace gbsp {

constexpr unsigned FULL = 0xffffffffu;

// Records a failure for gbsp_get_last_error / gbsp_last_error_message and returns status.
int fail(int status, const char *fmt, ...);
// Clears the per-thread error record and returns GBSP_OK.
int ok();
// Adds n to the process-wide count of kernels launched by the library.
void count_launches(int n);
// Converts a pending launch error into GBSP_ERR_CUDA (with the CUDA message).
int check_launch(const char *what);
// Fault selected by the GBSP_FAULT environment variable (0 none, 1 alloc, 2 launch, 3 validate).
int injected_fault();
// SM count of the current device (cached per device).
int sm_count();
// Stream-ordered scratch from a library-owned pool that keeps its memory between calls.
int scratch_alloc(void **ptr, size_t bytes, cudaStream_t s);
void scratch_free(void *ptr, cudaStream_t s);

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ---- element types ----------------------------------------------------------------------
// Each dense element type is read 16 bytes at a time (one 128-bit load per lane): V
// elements per vector.  A-values of the same type give one FP32 coefficient per nonzero.

struct F32 {
    using stored = float;
    static constexpr int V = 4;
    static constexpr int dtype = GBSP_F32;
    __device__ __forceinline__ static void unpack(const uint4 &r, float (&o)[4]) {
        o[0] = __uint_as_float(r.x);
        o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z);
        o[3] = __uint_as_float(r.w);
    }
    __device__ __forceinline__ static float value(float v) { return v; }
    __device__ __forceinline__ static float scalar(const stored *p) { return *p; }
    // acc[k] += a * element k of the vector r (single-rounding fmaf per element)
    __device__ __forceinline__ static void axpy(float a, const uint4 &r, float (&acc)[4]) {
        float o[4];
        unpack(r, o);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fmaf(a, o[k], acc[k]);
    }
    // sum + <x, y> over one vector, element by element in order (x decoded as xf, packed as xr)
    __device__ __forceinline__ static float dot(const uint4 &xr, const float (&xf)[4], const uint4 &yr, float sum) {
        float y[4];
        unpack(yr, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) sum = fmaf(xf[k], y[k], sum);
        return sum;
    }
};

struct BF16 {
    using stored = uint16_t;
    static constexpr int V = 8;
    static constexpr int dtype = GBSP_BF16;
    __device__ __forceinline__ static void unpack(const uint4 &r, float (&o)[8]) {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = __uint_as_float(w[i] << 16);
            o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static float value(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
    __device__ __forceinline__ static float scalar(const stored *p) { return value(*p); }
    // acc[k] += a * element k of the vector r, where a must hold a BF16 value (its low 16
    // bits zero; every BF16-form coefficient is an A value decoded from BF16).  The product
    // of two BF16 values is exact in FP32, so the mixed-precision fma (BF16 multiplicands,
    // FP32 addend and result, one rounding) gives exactly fmaf of the decoded values,
    // without decoding the eight elements first.
    __device__ __forceinline__ static void axpy(float a, const uint4 &r, float (&acc)[8]) {
        const uint32_t ab = __float_as_uint(a) >> 16;
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm("{\n\t.reg .b16 al, ah, bl, bh;\n\t"
                "mov.b32 {al, ah}, %2;\n\t"
                "mov.b32 {bl, bh}, %3;\n\t"
                "fma.rn.f32.bf16 %0, al, bl, %0;\n\t"
                "fma.rn.f32.bf16 %1, al, bh, %1;\n\t}"
                : "+f"(acc[2 * i]), "+f"(acc[2 * i + 1])
                : "r"(ab), "r"(w[i]));
    }
    // sum + <x, y> over one vector, element by element in order, with the mixed-precision
    // fma on the packed BF16 elements of x and y (exact products, as fmaf of decoded values)
    __device__ __forceinline__ static float dot(const uint4 &xr, const float (&)[8], const uint4 &yr, float sum) {
        const uint32_t xw[4] = {xr.x, xr.y, xr.z, xr.w}, yw[4] = {yr.x, yr.y, yr.z, yr.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm("{\n\t.reg .b16 xl, xh, yl, yh;\n\t"
                "mov.b32 {xl, xh}, %1;\n\t"
                "mov.b32 {yl, yh}, %2;\n\t"
                "fma.rn.f32.bf16 %0, xl, yl, %0;\n\t"
                "fma.rn.f32.bf16 %0, xh, yh, %0;\n\t}"
                : "+f"(sum)
                : "r"(xw[i]), "r"(yw[i]));
        return sum;
    }
};

struct E4M3 {
    using stored = uint8_t;
    static constexpr int V = 16;
    static constexpr int dtype = GBSP_E4M3;
    __device__ __forceinline__ static float2 pair(uint16_t two) {
        __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)two, __NV_E4M3);
        return __half22float2(*reinterpret_cast<__half2 *>(&h));
    }
    __device__ __forceinline__ static void unpack(const uint4 &r, float (&o)[16]) {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 a = pair((uint16_t)(w[i] & 0xffffu));
            float2 b = pair((uint16_t)(w[i] >> 16));
            o[4 * i] = a.x;
            o[4 * i + 1] = a.y;
            o[4 * i + 2] = b.x;
            o[4 * i + 3] = b.y;
        }
    }
    __device__ __forceinline__ static float value(uint8_t q) {
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&h));
    }
    __device__ __forceinline__ static float scalar(const stored *p) { return value(*p); }
    __device__ __forceinline__ static void axpy(float a, const uint4 &r, float (&acc)[16]) {
        float o[16];
        unpack(r, o);
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = fmaf(a, o[k], acc[k]);
    }
    __device__ __forceinline__ static float dot(const uint4 &, const float (&xf)[16], const uint4 &yr, float sum) {
        float y[16];
        unpack(yr, y);
#pragma unroll
        for (int k = 0; k < 16; ++k) sum = fmaf(xf[k], y[k], sum);
        return sum;
    }
};

// Streaming (read-once) loads: indices and values are touched once, so keep them from
// displacing the gathered dense rows in L1 / L2.
__device__ __forceinline__ int ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ uint16_t ld_stream(const uint16_t *p) { return __ldcs(reinterpret_cast<const unsigned short *>(p)); }
__device__ __forceinline__ uint8_t ld_stream(const uint8_t *p) { return __ldcs(reinterpret_cast<const unsigned char *>(p)); }

// Packed FP32 arithmetic (FFMA2 on sm_100+): two independent single-rounding fmas per
// instruction.  axpy2 gives every element exactly what fmaf gives it; dot2 keeps two
// running sums (even and odd elements), added at the end.  Used where instruction issue
// binds (the graph chain, the entry-split SDDMM on short rows); measured on the same GPU,
// the L2-bound row-split SpMM / SDDMM kernels ran 5-14% slower with it at N = Kd = 256, so
// they keep scalar fmaf.
template <int V>
__device__ __forceinline__ void axpy2(float a, const float (&b)[V], float (&acc)[V]) {
    static_assert(V % 2 == 0, "pairs");
#pragma unroll
    for (int k = 0; k < V; k += 2) {
        const float2 r = __ffma2_rn(make_float2(a, a), make_float2(b[k], b[k + 1]), make_float2(acc[k], acc[k + 1]));
        acc[k] = r.x;
        acc[k + 1] = r.y;
    }
}
template <int V>
__device__ __forceinline__ void dot2(const float (&x)[V], const float (&y)[V], float2 &acc) {
    static_assert(V % 2 == 0, "pairs");
#pragma unroll
    for (int k = 0; k < V; k += 2) acc = __ffma2_rn(make_float2(x[k], x[k + 1]), make_float2(y[k], y[k + 1]), acc);
}

// Two adjacent 16-byte vectors of a gathered row with one 32-byte load (read-only path, L1
// cached like ld_gather16); p must be 32-byte aligned.
__device__ __forceinline__ void ld_gather32(const void *p, uint4 &a, uint4 &b) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}
inline bool aligned32(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 31u) == 0; }

// Gathered dense rows: read-only path, 16 bytes per lane.  (Skipping L1 allocation for
// them measured 1-9% slower on the 65,536^2 and 16,384^2 workloads, so they stay cached.)
__device__ __forceinline__ uint4 ld_gather16(const void *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// Merge-path coordinate of diagonal d over the two lists "row ends" (rowptr[1..M]) and
// "stored entries" (0..nnz-1): the number x of rows fully consumed, with y = d - x
// entries consumed.  Row end i precedes entry j exactly when rowptr[i + 1] <= j.
// The warp evaluates 32 probes per round (a 33-ary search), then settles the last <= 32.
__device__ __forceinline__ int merge_search(const int32_t *rowptr, int M, int64_t nnz, int64_t d, int lane) {
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < M ? d : M;
    while (hi - lo > 32) {
        const int64_t span = hi - lo;
        const int64_t probe = lo + (span * (lane + 1)) / 33;
        const bool t = (int64_t)__ldg(rowptr + probe + 1) + probe + 1 <= d;
        const int k = __popc(__ballot_sync(FULL, t));
        const int64_t new_lo = k == 0 ? lo : lo + (span * k) / 33 + 1;
        const int64_t new_hi = k == 32 ? hi : lo + (span * (k + 1)) / 33;
        lo = new_lo;
        hi = new_hi;
    }
    const int64_t x = lo + lane;
    const bool t = x < hi && (int64_t)__ldg(rowptr + x + 1) + x + 1 <= d;
    return (int)(lo + __popc(__ballot_sync(FULL, t)));
}

// ---- launch descriptors -------------------------------------------------------------------

struct SpmmProblem {
    int32_t M, K, N;
    int64_t nnz;  // -1 when the caller did not say (read on the device where needed)
    const int32_t *rowptr, *colidx;
    const void *vals;
    const float *a_scale;  // E4M3 per-row scale of A (s_i), else null
    const void *B;
    int64_t ldb;
    const float *b_scale;  // E4M3 per-row scale of B (t_k), else null
    float *C;
    int64_t ldc;
    int dtype;
};

struct SddmmProblem {
    int32_t M, N, Kd;
    int64_t nnz;
    const int32_t *rowptr, *colidx;
    const float *svals;
    const void *X;
    int64_t ldx;
    const float *x_scale;
    const void *Y;
    int64_t ldy;
    const float *y_scale;
    float *out;
    int dtype;  // dtype of X and Y
    const int32_t *pos;  // row split only: entry e's value and output at pos[e] (null: at e)
};

// SpMM launchers: one translation unit per (element type, algorithm).
template <class EL, int ALGO>
int launch_spmm_algo(const SpmmProblem &p, int vecs, int unroll, int ctas_per_sm, cudaStream_t s);
template <class EL>
int launch_sddmm_typed(const SddmmProblem &p, int variant, int vecs, cudaStream_t s);

// vecs: 16-byte vectors per lane (0 = default); unroll: gathers in flight per lane.
int launch_spmm(const SpmmProblem &p, int variant, int vecs, int unroll, int ctas_per_sm, cudaStream_t s);
int launch_sddmm(const SddmmProblem &p, int variant, int vecs, cudaStream_t s);
int launch_validate(const gbsp_csr &A, unsigned long long *d_count, cudaStream_t s);
// The split GBSP_VARIANT_AUTO takes for op on A's pattern, from row statistics measured
// on the first call (synchronising) and re-measured asynchronously on later ones; stats
// receives {rows, nnz, sum of squared lengths, longest row, empty rows} when non-null.
// b_bytes and row_bytes describe the gathered dense operand (B of SpMM, Y of SDDMM).
constexpr int kOpSpmm = 0, kOpSddmm = 1;
int auto_choice(const gbsp_csr &A, int op, int64_t b_bytes, int64_t row_bytes, cudaStream_t s, int *variant,
                int64_t *stats);
int auto_spmm_rule(int64_t M, int64_t nnz, int64_t sumsq, int64_t maxlen, int64_t b_bytes, int64_t row_bytes);
int auto_sddmm_rule(int64_t M, int64_t nnz, int64_t sumsq, int64_t maxlen, int64_t y_bytes, int64_t row_bytes);
void auto_forget_all();
int launch_quant_bf16(const float *x, uint16_t *out, int64_t n, cudaStream_t s);
int launch_quant_e4m3_rows(const float *x, const int32_t *rowptr, int64_t nrows, int64_t ncols,
                           int64_t ld, uint8_t *q, float *scale, cudaStream_t s);

}  // namespace gbsp

// C ABI entry points: argument checks, variant choice and dispatch to the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace gbsp {

namespace {
thread_local int t_status = GBSP_OK;
thread_local char t_msg[512] = "";
std::mutex g_mu;
std::atomic<long long> g_launches{0};
int g_sm[64] = {0};
cudaMemPool_t g_pool[64] = {nullptr};
}  // namespace

int fail(int status, const char *fmt, ...) {
    t_status = status;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_msg, sizeof t_msg, fmt, ap);
    va_end(ap);
    return status;
}

int ok() {
    t_status = GBSP_OK;
    t_msg[0] = 0;
    return GBSP_OK;
}

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Host-side fault injection for testing the error paths without touching the GPU:
// GBSP_FAULT=alloc makes workspace allocation fail, =launch makes the SpMM / SDDMM entry
// points fail before launching, =validate makes gbsp_csr_validate report a bad matrix.
int injected_fault() {
    static int f = [] {
        const char *e = getenv("GBSP_FAULT");
        if (!e) return 0;
        if (!strcmp(e, "alloc")) return 1;
        if (!strcmp(e, "launch")) return 2;
        if (!strcmp(e, "validate")) return 3;
        return 0;
    }();
    return f;
}

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GBSP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GBSP_OK;
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (g_sm[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sm[dev] = n;
    }
    return g_sm[dev];
}

int scratch_alloc(void **ptr, size_t bytes, cudaStream_t s) {
    if (injected_fault() == 1) {
        *ptr = nullptr;
        return fail(GBSP_ERR_OOM, "injected workspace allocation failure (GBSP_FAULT=alloc)");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(GBSP_ERR_CUDA, "no current device");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) {
                g_pool[dev] = nullptr;
                cudaGetLastError();
                return fail(GBSP_ERR_OOM, "workspace pool creation failed");
            }
            uint64_t keep = UINT64_MAX;  // keep freed workspace for the next call
            cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (cudaMallocFromPoolAsync(ptr, bytes ? bytes : 16, g_pool[dev], s) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(GBSP_ERR_OOM, "workspace of %zu bytes could not be allocated", bytes);
    }
    return GBSP_OK;
}

void scratch_free(void *ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}

int launch_sddmm(const SddmmProblem &p, int variant, int vecs, cudaStream_t s) {
    switch (p.dtype) {
        case GBSP_F32: return launch_sddmm_typed<F32>(p, variant, vecs, s);
        case GBSP_BF16: return launch_sddmm_typed<BF16>(p, variant, vecs, s);
        case GBSP_E4M3: return launch_sddmm_typed<E4M3>(p, variant, vecs, s);
    }
    return fail(GBSP_ERR_UNSUPPORTED, "sddmm: dtype %d", p.dtype);
}

namespace {

constexpr int64_t kMax32 = 2147483647LL;

int elem_bytes(int dtype) { return dtype == GBSP_F32 ? 4 : dtype == GBSP_BF16 ? 2 : dtype == GBSP_E4M3 ? 1 : 0; }
int elems_per_vec(int dtype) { return 16 / elem_bytes(dtype); }

int check_csr(const gbsp_csr *A, const char *who) {
    if (!A) return fail(GBSP_ERR_INVALID_ARG, "%s: null CSR descriptor", who);
    if (A->rows < 0 || A->cols < 0 || A->rows > kMax32 || A->cols > kMax32 || A->nnz > kMax32 || A->nnz < -1)
        return fail(GBSP_ERR_INVALID_ARG, "%s: CSR sizes out of range", who);
    if (A->rows > 0 && !A->rowptr) return fail(GBSP_ERR_INVALID_ARG, "%s: null rowptr", who);
    if (A->nnz != 0 && (!A->colidx || !A->vals)) return fail(GBSP_ERR_INVALID_ARG, "%s: null colidx / vals", who);
    if (elem_bytes(A->dtype) == 0) return fail(GBSP_ERR_INVALID_ARG, "%s: bad CSR dtype", who);
    return GBSP_OK;
}

int check_dense(const gbsp_dense *D, const char *who, const char *name) {
    if (!D) return fail(GBSP_ERR_INVALID_ARG, "%s: null %s descriptor", who, name);
    if (D->rows < 0 || D->cols < 0 || D->rows > kMax32 || D->cols > kMax32 || D->ld < D->cols)
        return fail(GBSP_ERR_INVALID_ARG, "%s: %s sizes out of range (ld must be >= cols)", who, name);
    if (D->rows > 0 && D->cols > 0 && !D->data) return fail(GBSP_ERR_INVALID_ARG, "%s: null %s data", who, name);
    if (elem_bytes(D->dtype) == 0) return fail(GBSP_ERR_INVALID_ARG, "%s: bad %s dtype", who, name);
    if (D->dtype == GBSP_E4M3 && D->rows > 0 && !D->row_scale)
        return fail(GBSP_ERR_INVALID_ARG, "%s: E4M3 %s needs row scales", who, name);
    return GBSP_OK;
}

bool vec_ok(const gbsp_dense *D) {
    const int V = elems_per_vec(D->dtype);
    return aligned16(D->data) && D->ld % V == 0 && D->cols % V == 0;
}

}  // namespace
}  // namespace gbsp

using namespace gbsp;

GBSP_EXPORT int spmm_csr_ex(const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, const gbsp_opts *opts,
                            void *stream) {
    int st;
    if ((st = check_csr(A, "spmm")) || (st = check_dense(B, "spmm", "B")) || (st = check_dense(C, "spmm", "C")))
        return st;
    if (B->rows != A->cols || C->rows != A->rows || C->cols != B->cols)
        return fail(GBSP_ERR_INVALID_ARG, "spmm: shape mismatch A %lldx%lld, B %lldx%lld, C %lldx%lld",
                    (long long)A->rows, (long long)A->cols, (long long)B->rows, (long long)B->cols,
                    (long long)C->rows, (long long)C->cols);
    if (A->dtype != B->dtype) return fail(GBSP_ERR_UNSUPPORTED, "spmm: A and B must have the same dtype");
    if (C->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "spmm: C must be FP32");
    if (A->dtype == GBSP_E4M3 && A->rows > 0 && !A->row_scale)
        return fail(GBSP_ERR_INVALID_ARG, "spmm: E4M3 A needs row scales");
    gbsp_opts o = opts ? *opts : gbsp_opts{};
    if (o.unroll != 0 && o.unroll != 1 && o.unroll != 2 && o.unroll != 4 && o.unroll != 8)
        return fail(GBSP_ERR_INVALID_ARG, "spmm: unroll must be 0, 1, 2, 4 or 8");
    if (o.vecs != 0 && o.vecs != 1 && o.vecs != 2 && o.vecs != 4)
        return fail(GBSP_ERR_INVALID_ARG, "spmm: vecs must be 0, 1, 2 or 4");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.validate && A->nnz >= 0) {
        int64_t bad = 0;
        if ((st = gbsp_csr_validate(A, stream, &bad))) return st;
    }
    if (A->rows == 0 || B->cols == 0) return ok();
    if (injected_fault() == 2) return fail(GBSP_ERR_CUDA, "spmm: injected launch failure (GBSP_FAULT=launch)");
    const bool vec = vec_ok(B) && aligned16(C->data) && C->ld % 4 == 0;
    int variant = o.variant;
    if (variant == GBSP_VARIANT_AUTO) {
        variant = GBSP_VARIANT_SCALAR;
        const int64_t rb = B->cols * elem_bytes(B->dtype);
        if (vec && (st = auto_choice(*A, kOpSpmm, B->rows * rb, rb, s, &variant, nullptr))) return st;
    }
    if (variant != GBSP_VARIANT_SCALAR && !vec)
        return fail(GBSP_ERR_ALIGN, "spmm: vectorised variant needs 16-byte aligned B and C, and N and ld "
                                    "multiples of %d", elems_per_vec(B->dtype));
    if (variant == GBSP_VARIANT_ENTRY)
        return fail(GBSP_ERR_UNSUPPORTED, "spmm: the entry split is an SDDMM variant (SpMM rows need one owner)");
    if (variant == GBSP_VARIANT_HSP_PLAN || variant == GBSP_VARIANT_SELL_PLAN)
        return fail(GBSP_ERR_UNSUPPORTED, "spmm: the hyper-sparse and SELL-C-sigma plans run through their own "
                                          "plan entry points");
    if (variant < GBSP_VARIANT_ROWSPLIT || variant > GBSP_VARIANT_ROWGROUP)
        return fail(GBSP_ERR_INVALID_ARG, "spmm: unknown variant %d", variant);
    SpmmProblem p{};
    p.M = (int32_t)A->rows;
    p.K = (int32_t)A->cols;
    p.N = (int32_t)B->cols;
    p.nnz = A->nnz;
    p.rowptr = A->rowptr;
    p.colidx = A->colidx;
    p.vals = A->vals;
    p.a_scale = A->row_scale;
    p.B = B->data;
    p.ldb = B->ld;
    p.b_scale = B->row_scale;
    p.C = static_cast<float *>(C->data);
    p.ldc = C->ld;
    p.dtype = A->dtype;
    if ((st = launch_spmm(p, variant, o.vecs, o.unroll, o.ctas_per_sm, s))) return st;
    return ok();
}

GBSP_EXPORT int sddmm_csr_ex(const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y, float *out,
                             const gbsp_opts *opts, void *stream) {
    int st;
    if ((st = check_csr(S, "sddmm")) || (st = check_dense(X, "sddmm", "X")) || (st = check_dense(Y, "sddmm", "Y")))
        return st;
    if (X->rows != S->rows || Y->rows != S->cols || X->cols != Y->cols)
        return fail(GBSP_ERR_INVALID_ARG, "sddmm: shape mismatch S %lldx%lld, X %lldx%lld, Y %lldx%lld",
                    (long long)S->rows, (long long)S->cols, (long long)X->rows, (long long)X->cols,
                    (long long)Y->rows, (long long)Y->cols);
    if (S->dtype != GBSP_F32) return fail(GBSP_ERR_UNSUPPORTED, "sddmm: S values must be FP32");
    if (X->dtype != Y->dtype) return fail(GBSP_ERR_UNSUPPORTED, "sddmm: X and Y must have the same dtype");
    if (S->nnz != 0 && !out) return fail(GBSP_ERR_INVALID_ARG, "sddmm: null out");
    gbsp_opts o = opts ? *opts : gbsp_opts{};
    if (o.vecs != 0 && o.vecs != 1 && o.vecs != 2 && o.vecs != 4)
        return fail(GBSP_ERR_INVALID_ARG, "sddmm: vecs must be 0, 1, 2 or 4");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.validate && S->nnz >= 0) {
        int64_t bad = 0;
        if ((st = gbsp_csr_validate(S, stream, &bad))) return st;
    }
    if (S->rows == 0 || S->nnz == 0) return ok();
    if (injected_fault() == 2) return fail(GBSP_ERR_CUDA, "sddmm: injected launch failure (GBSP_FAULT=launch)");
    const int V = elems_per_vec(X->dtype);
    const bool vec = vec_ok(X) && vec_ok(Y) && X->cols > 0 && X->cols <= 32 * 16;
    int variant = o.variant;
    if (variant == GBSP_VARIANT_AUTO) {
        variant = GBSP_VARIANT_SCALAR;
        const int64_t rb = Y->cols * elem_bytes(Y->dtype);
        if (vec && (st = auto_choice(*S, kOpSddmm, Y->rows * rb, rb, s, &variant, nullptr))) return st;
    }
    if (variant != GBSP_VARIANT_SCALAR && !vec)
        return fail(GBSP_ERR_ALIGN, "sddmm: vectorised variant needs 16-byte aligned X and Y, Kd and ld "
                                    "multiples of %d and Kd <= %d", V, 32 * 16);
    if (variant == GBSP_VARIANT_ROWGROUP || variant == GBSP_VARIANT_HSP_PLAN || variant == GBSP_VARIANT_SELL_PLAN)
        return fail(GBSP_ERR_UNSUPPORTED, "sddmm: the row groups and the SpMM plans are SpMM variants");
    if (variant < GBSP_VARIANT_ROWSPLIT || variant > GBSP_VARIANT_ENTRY)
        return fail(GBSP_ERR_INVALID_ARG, "sddmm: unknown variant %d", variant);
    SddmmProblem p{};
    p.M = (int32_t)S->rows;
    p.N = (int32_t)S->cols;
    p.Kd = (int32_t)X->cols;
    p.nnz = S->nnz;
    p.rowptr = S->rowptr;
    p.colidx = S->colidx;
    p.svals = static_cast<const float *>(S->vals);
    p.X = X->data;
    p.ldx = X->ld;
    p.x_scale = X->row_scale;
    p.Y = Y->data;
    p.ldy = Y->ld;
    p.y_scale = Y->row_scale;
    p.out = out;
    p.dtype = X->dtype;
    if ((st = launch_sddmm(p, variant, o.vecs, s))) return st;
    return ok();
}

GBSP_EXPORT int spmm_csr(const int32_t *rowptr, const int32_t *colidx, const float *vals, const float *B, float *C,
                         int64_t M, int64_t K, int64_t N) {
    gbsp_csr A{M, K, -1, rowptr, colidx, vals, nullptr, GBSP_F32};
    gbsp_dense b{const_cast<float *>(B), K, N, N, nullptr, GBSP_F32};
    gbsp_dense c{C, M, N, N, nullptr, GBSP_F32};
    if (M > 0 && (!colidx || !vals)) return fail(GBSP_ERR_INVALID_ARG, "spmm_csr: null colidx / vals");
    return spmm_csr_ex(&A, &b, &c, nullptr, nullptr);
}

GBSP_EXPORT int sddmm_csr(const int32_t *rowptr, const int32_t *colidx, const float *svals, const float *X,
                          const float *Y, float *out, int64_t M, int64_t N, int64_t Kd) {
    gbsp_csr S{M, N, -1, rowptr, colidx, svals, nullptr, GBSP_F32};
    gbsp_dense x{const_cast<float *>(X), M, Kd, Kd, nullptr, GBSP_F32};
    gbsp_dense y{const_cast<float *>(Y), N, Kd, Kd, nullptr, GBSP_F32};
    if (M > 0 && (!colidx || !svals || !out)) return fail(GBSP_ERR_INVALID_ARG, "sddmm_csr: null pointer");
    return sddmm_csr_ex(&S, &x, &y, out, nullptr, nullptr);
}

GBSP_EXPORT int gbsp_csr_validate(const gbsp_csr *A, void *stream, int64_t *n_bad) {
    int st;
    if ((st = check_csr(A, "validate"))) return st;
    if (!n_bad) return fail(GBSP_ERR_INVALID_ARG, "validate: null n_bad");
    if (A->nnz < 0) return fail(GBSP_ERR_INVALID_ARG, "validate: nnz must be given");
    if (injected_fault() == 3) {
        *n_bad = -1;
        return fail(GBSP_ERR_INVALID_CSR, "validate: injected failure (GBSP_FAULT=validate)");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *d = nullptr;
    if ((st = scratch_alloc(&d, sizeof(unsigned long long), s))) return st;
    unsigned long long h = 0;
    st = launch_validate(*A, static_cast<unsigned long long *>(d), s);
    if (st == GBSP_OK) {
        if (cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = check_launch("validate copy");
    }
    scratch_free(d, s);
    if (st) return st;
    *n_bad = (int64_t)h;
    if (h) return fail(GBSP_ERR_INVALID_CSR, "validate: %llu violations", h);
    return ok();
}

GBSP_EXPORT int gbsp_quantize_bf16(const float *x, uint16_t *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return fail(GBSP_ERR_INVALID_ARG, "quantize_bf16: bad arguments");
    if (n == 0) return ok();
    int st = launch_quant_bf16(x, out, n, static_cast<cudaStream_t>(stream));
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_quantize_e4m3_rows(const float *x, const int32_t *rowptr, int64_t nrows, int64_t ncols,
                                        int64_t ld, uint8_t *q, float *scale, void *stream) {
    if (nrows < 0 || nrows > kMax32 || (!rowptr && (ncols < 0 || ld < ncols)))
        return fail(GBSP_ERR_INVALID_ARG, "quantize_e4m3_rows: bad sizes");
    if (nrows > 0 && (!scale || (!rowptr && ncols > 0 && (!x || !q))))
        return fail(GBSP_ERR_INVALID_ARG, "quantize_e4m3_rows: null pointer");
    if (nrows == 0) return ok();
    int st = launch_quant_e4m3_rows(x, rowptr, nrows, ncols, ld, q, scale, static_cast<cudaStream_t>(stream));
    return st ? st : ok();
}

GBSP_EXPORT const char *gbsp_status_string(int status) {
    switch (status) {
        case GBSP_OK: return "ok";
        case GBSP_ERR_INVALID_ARG: return "invalid argument";
        case GBSP_ERR_INVALID_CSR: return "invalid CSR";
        case GBSP_ERR_ALIGN: return "operand alignment not supported by the requested variant";
        case GBSP_ERR_UNSUPPORTED: return "unsupported combination";
        case GBSP_ERR_CUDA: return "CUDA error";
        case GBSP_ERR_OOM: return "out of device memory";
        case GBSP_ERR_TIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

GBSP_EXPORT int gbsp_get_last_error(void) { return t_status; }
GBSP_EXPORT const char *gbsp_last_error_message(void) { return t_msg; }
GBSP_EXPORT int gbsp_device_sm_count(void) { return sm_count(); }
GBSP_EXPORT int64_t gbsp_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

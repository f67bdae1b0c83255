// Host-resident SpMM / SDDMM: the CSR streams to the device in row chunks while earlier
// chunks compute and their results stream back, the GPU counterpart of the paper's
// streamed A with results copied back per chunk (Section III-A) and of its overlap of
// transfers with computation (Section III-A-2, multiple accumulator rows).
//
// Three streams: host-to-device copies, kernels, device-to-host copies.  Each chunk of
// rows goes through one of `slots` device buffers (row pointers, column indices, values,
// its C rows and its SDDMM outputs); events order copy -> compute -> copy-back per chunk,
// and a slot is refilled only after its previous chunk's results have left the device.  The
// gathered dense operands (B for SpMM, Y for SDDMM) are copied once at the start; the rows
// of X travel with their chunk.  Column
// indices and values of chunk [r0, r1) sit at device offset 0 while the kernels index
// them with the matrix's absolute entry numbers, so the kernels get base pointers moved
// back by rowptr[r0].
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace gbsp {
namespace {

struct Slot {
    int32_t *rowptr = nullptr, *colidx = nullptr;
    float *vals = nullptr, *C = nullptr, *out = nullptr;
    cudaEvent_t copied = nullptr, computed = nullptr, drained = nullptr;
};

// The streams and events of the pipeline, created once per host thread and device and
// reused by every call (calls from one thread are ordered through the caller's stream, so
// they never use them concurrently).
struct Executor {
    int device = -1;
    cudaStream_t in = nullptr, run = nullptr, out = nullptr;
    cudaEvent_t ready = nullptr, dense_in = nullptr, all_out = nullptr;
    std::vector<Slot> slots;  // events only; buffers are taken per call

    int prepare(int dev, int nslots) {
        if (device != dev) {
            release();
            device = dev;
            if (cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&run, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&dense_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&all_out, cudaEventDisableTiming) != cudaSuccess) {
                release();
                return check_launch("host pipeline streams");
            }
        }
        while ((int)slots.size() < nslots) {
            Slot x;
            if (cudaEventCreateWithFlags(&x.copied, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&x.computed, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&x.drained, cudaEventDisableTiming) != cudaSuccess)
                return check_launch("host pipeline events");
            slots.push_back(x);
        }
        return GBSP_OK;
    }
    void release() {
        for (auto &x : slots) {
            if (x.copied) cudaEventDestroy(x.copied);
            if (x.computed) cudaEventDestroy(x.computed);
            if (x.drained) cudaEventDestroy(x.drained);
        }
        slots.clear();
        for (cudaEvent_t e : {ready, dense_in, all_out})
            if (e) cudaEventDestroy(e);
        for (cudaStream_t t : {in, run, out})
            if (t) cudaStreamDestroy(t);
        in = run = out = nullptr;
        ready = dense_in = all_out = nullptr;
        device = -1;
    }
};

}  // namespace
}  // namespace gbsp

using namespace gbsp;

GBSP_EXPORT int gbsp_spmm_sddmm_host(const int32_t *rowptr, const int32_t *colidx, const float *vals,
                                     const float *B, float *C, int64_t N, const float *X, const float *Y,
                                     float *out, int64_t Kd, int64_t M, int64_t K, int64_t nnz, int32_t chunks,
                                     int32_t slots, void *stream) {
    const bool do_spmm = B && C && N > 0, do_sddmm = X && Y && out && Kd > 0;
    if (M < 0 || K < 0 || nnz < 0 || M > 2147483647LL || K > 2147483647LL || nnz > 2147483647LL ||
        (M > 0 && !rowptr) || (nnz > 0 && (!colidx || !vals)) || N < 0 || Kd < 0)
        return fail(GBSP_ERR_INVALID_ARG, "host pipeline: bad arguments");
    if (!do_spmm && !do_sddmm) return ok();
    if ((do_spmm && N % 4) || (do_sddmm && Kd % 4))
        return fail(GBSP_ERR_ALIGN, "host pipeline: N and Kd must be multiples of 4");
    if (M == 0) return ok();
    if (chunks < 1) chunks = 8;
    if (chunks > M) chunks = (int32_t)M;
    if (slots < 2) slots = 2;
    if (slots > chunks) slots = chunks;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    // chunk boundaries: the first c chunks hold a fraction 1 - (1 - c / chunks)^1.5 of the
    // entries, so chunks shrink toward the end and the last chunk's compute and copy-back,
    // which nothing overlaps, stay short
    std::vector<int64_t> bounds(1, 0);
    for (int c = 1; c < chunks; ++c) {
        const double rest = 1.0 - (double)c / chunks;
        const int64_t want = (int64_t)((double)nnz * (1.0 - rest * std::sqrt(rest)));
        int64_t lo = bounds.back() + 1, hi = M - (chunks - c);
        while (lo < hi) {  // first row whose start reaches `want`
            const int64_t mid = (lo + hi) / 2;
            if (rowptr[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        bounds.push_back(lo);
    }
    bounds.push_back(M);
    int64_t max_rows = 0, max_nnz = 0;
    for (int c = 0; c < chunks; ++c) {
        max_rows = std::max(max_rows, bounds[c + 1] - bounds[c]);
        max_nnz = std::max(max_nnz, (int64_t)(rowptr[bounds[c + 1]] - rowptr[bounds[c]]));
    }
    static thread_local Executor ex;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_launch("host pipeline device");
    int st = ex.prepare(dev, slots);
    if (st) return st;
    cudaStream_t s_in = ex.in, s_run = ex.run, s_out = ex.out;
    cudaEvent_t ready = ex.ready, dense_in = ex.dense_in, all_out = ex.all_out;
    std::vector<Slot> sl(ex.slots.begin(), ex.slots.begin() + slots);
    void *dB = nullptr, *dX = nullptr, *dY = nullptr;
#define GBSP_CU(x)                                                             \
    do {                                                                       \
        if ((x) != cudaSuccess && st == GBSP_OK) st = check_launch("host pipeline"); \
    } while (0)
    // everything starts after the work already queued on the caller's stream
    GBSP_CU(cudaEventRecord(ready, user));
    GBSP_CU(cudaStreamWaitEvent(s_in, ready, 0));
    for (auto &x : sl) {
        if (scratch_alloc((void **)&x.rowptr, sizeof(int32_t) * (size_t)(max_rows + 1), s_in) ||
            scratch_alloc((void **)&x.colidx, sizeof(int32_t) * (size_t)std::max<int64_t>(max_nnz, 1), s_in) ||
            scratch_alloc((void **)&x.vals, sizeof(float) * (size_t)std::max<int64_t>(max_nnz, 1), s_in) ||
            (do_spmm && scratch_alloc((void **)&x.C, sizeof(float) * (size_t)(max_rows * N), s_in)) ||
            (do_sddmm && scratch_alloc((void **)&x.out, sizeof(float) * (size_t)std::max<int64_t>(max_nnz, 1), s_in))) {
            st = GBSP_ERR_OOM;
            goto done;
        }
    }
    if (do_spmm && scratch_alloc(&dB, sizeof(float) * (size_t)(K * N), s_in)) st = GBSP_ERR_OOM;
    if (!st && do_sddmm &&
        (scratch_alloc(&dX, sizeof(float) * (size_t)(M * Kd), s_in) ||
         scratch_alloc(&dY, sizeof(float) * (size_t)(K * Kd), s_in)))
        st = GBSP_ERR_OOM;
    if (st) goto done;
    if (do_spmm) GBSP_CU(cudaMemcpyAsync(dB, B, sizeof(float) * (size_t)(K * N), cudaMemcpyHostToDevice, s_in));
    if (do_sddmm) GBSP_CU(cudaMemcpyAsync(dY, Y, sizeof(float) * (size_t)(K * Kd), cudaMemcpyHostToDevice, s_in));
    GBSP_CU(cudaEventRecord(dense_in, s_in));
    GBSP_CU(cudaStreamWaitEvent(s_run, dense_in, 0));
    for (int c = 0; c < chunks && !st; ++c) {
        Slot &x = sl[c % slots];
        const int64_t r0 = bounds[c], r1 = bounds[c + 1], mr = r1 - r0;
        const int64_t p0 = rowptr[r0], p1 = rowptr[r1], ne = p1 - p0;
        if (c >= slots) GBSP_CU(cudaStreamWaitEvent(s_in, x.drained, 0));  // slot's previous results are out
        GBSP_CU(cudaMemcpyAsync(x.rowptr, rowptr + r0, sizeof(int32_t) * (size_t)(mr + 1), cudaMemcpyHostToDevice, s_in));
        if (do_sddmm)  // X rows of the chunk, into the full-size X buffer (never reused)
            GBSP_CU(cudaMemcpyAsync(static_cast<float *>(dX) + r0 * Kd, X + r0 * Kd, sizeof(float) * (size_t)(mr * Kd),
                                    cudaMemcpyHostToDevice, s_in));
        if (ne > 0) {
            GBSP_CU(cudaMemcpyAsync(x.colidx, colidx + p0, sizeof(int32_t) * (size_t)ne, cudaMemcpyHostToDevice, s_in));
            GBSP_CU(cudaMemcpyAsync(x.vals, vals + p0, sizeof(float) * (size_t)ne, cudaMemcpyHostToDevice, s_in));
        }
        GBSP_CU(cudaEventRecord(x.copied, s_in));
        GBSP_CU(cudaStreamWaitEvent(s_run, x.copied, 0));
        if (do_spmm) {
            SpmmProblem p{};
            p.M = (int32_t)mr;
            p.K = (int32_t)K;
            p.N = (int32_t)N;
            p.nnz = ne;
            p.rowptr = x.rowptr;
            p.colidx = x.colidx - p0;  // absolute entry numbers index the chunk buffer
            p.vals = x.vals - p0;
            p.B = dB;
            p.ldb = N;
            p.C = x.C;
            p.ldc = N;
            p.dtype = GBSP_F32;
            if ((st = launch_spmm(p, GBSP_VARIANT_ROWSPLIT, 0, 0, 0, s_run))) break;
        }
        if (do_sddmm && ne > 0) {
            SddmmProblem q{};
            q.M = (int32_t)mr;
            q.N = (int32_t)K;
            q.Kd = (int32_t)Kd;
            q.nnz = ne;
            q.rowptr = x.rowptr;
            q.colidx = x.colidx - p0;
            q.svals = x.vals - p0;
            q.X = static_cast<const float *>(dX) + r0 * Kd;
            q.ldx = Kd;
            q.Y = dY;
            q.ldy = Kd;
            q.out = x.out - p0;
            q.dtype = GBSP_F32;
            if ((st = launch_sddmm(q, Kd <= 512 ? GBSP_VARIANT_ROWSPLIT : GBSP_VARIANT_SCALAR, 0, s_run))) break;
        }
        GBSP_CU(cudaEventRecord(x.computed, s_run));
        GBSP_CU(cudaStreamWaitEvent(s_out, x.computed, 0));
        if (do_spmm)
            GBSP_CU(cudaMemcpyAsync(C + r0 * N, x.C, sizeof(float) * (size_t)(mr * N), cudaMemcpyDeviceToHost, s_out));
        if (do_sddmm && ne > 0)
            GBSP_CU(cudaMemcpyAsync(out + p0, x.out, sizeof(float) * (size_t)ne, cudaMemcpyDeviceToHost, s_out));
        GBSP_CU(cudaEventRecord(x.drained, s_out));
    }
    // the caller's stream resumes after every result is on the host
    GBSP_CU(cudaEventRecord(all_out, s_out));
    GBSP_CU(cudaStreamWaitEvent(user, all_out, 0));
done:
#undef GBSP_CU
    for (auto &x : sl) {
        scratch_free(x.rowptr, s_out);
        scratch_free(x.colidx, s_out);
        scratch_free(x.vals, s_out);
        scratch_free(x.C, s_out);
        scratch_free(x.out, s_out);
    }
    scratch_free(dB, s_out);
    scratch_free(dX, s_out);
    scratch_free(dY, s_out);
    if (st) {  // leave the executor's streams idle for the next call
        cudaStreamSynchronize(s_in);
        cudaStreamSynchronize(s_run);
        cudaStreamSynchronize(s_out);
    }
    return st ? st : ok();
}

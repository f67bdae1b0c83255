// Automatic choice of the SpMM work split (GBSP_VARIANT_AUTO) from the row lengths of the
// sparsity pattern.
//
// Load balancing across rows of very different length is one of the GPU techniques the
// paper names for SpMM (Section II-D); which split wins depends on the row-length
// distribution, which the caller's CSR arrays do not state.  One integer pass over rowptr
// gives five counters (rows, stored entries, the sum of squared lengths, the longest row,
// empty rows), and a rule turns them into the split.  The first AUTO call on a pattern
// measures it and waits for the counters; the choice is kept in a small table keyed by
// (device, rowptr, colidx, rows, cols).  Every later call uses the kept choice and queues a
// new measurement whose counters land in pinned host memory; the call after it adopts them
// once they have arrived (an event query, never a wait).  So a different pattern that a
// caller puts at the same addresses (a caching allocator reuses them for arrays of the same
// size) gets its own choice from its second call on.  Only the choice is kept, never data
// derived from the pattern, so a stale choice costs speed, never correctness.  Under
// stream capture nothing is queued: a kept choice is used, else the row split.
#include <mutex>

#include "common.cuh"

namespace gbsp {
namespace {

// What a measurement delivers, into a pinned host slot mapped into the device's address
// space (so no copy follows the kernel).
struct StatsOut {
    unsigned long long sumsq, empty;
    unsigned int maxlen;
    int32_t nnz;
};
// A pattern's device accumulators: zero between measurements (the kernel's last block
// resets them after delivering).
struct StatsAcc {
    unsigned long long sumsq, empty;
    unsigned int maxlen, blocks_done;
};

// Grid-stride pass over the rows: per block, sum of squared lengths, empty rows and the
// longest row (integers, so the counters and the decision do not depend on the order),
// added into acc; the last block to finish writes the totals and rowptr[M] to out and
// clears acc for the next measurement.
__global__ void __launch_bounds__(256) row_stats_kernel(const int32_t *__restrict__ rowptr, int64_t M,
                                                        StatsAcc *acc, StatsOut *out) {
    unsigned long long sq = 0, empty = 0;
    unsigned int mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned int len = (unsigned int)(__ldg(rowptr + i + 1) - __ldg(rowptr + i));
        sq += (unsigned long long)len * len;
        empty += len == 0;
        mx = max(mx, len);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sq += __shfl_xor_sync(FULL, sq, off);
        empty += __shfl_xor_sync(FULL, empty, off);
        mx = max(mx, __shfl_xor_sync(FULL, mx, off));
    }
    __shared__ unsigned long long s_sq[8], s_empty[8];
    __shared__ unsigned int s_mx[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_sq[warp] = sq;
        s_empty[warp] = empty;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            sq += s_sq[w];
            empty += s_empty[w];
            mx = max(mx, s_mx[w]);
        }
        atomicAdd(&acc->sumsq, sq);
        atomicAdd(&acc->empty, empty);
        atomicMax(&acc->maxlen, mx);
        __threadfence();
        if (atomicAdd(&acc->blocks_done, 1u) == gridDim.x - 1) {  // every block's counters are in
            __threadfence();
            out->sumsq = atomicAdd(&acc->sumsq, 0ull);
            out->empty = atomicAdd(&acc->empty, 0ull);
            out->maxlen = atomicMax(&acc->maxlen, 0u);
            out->nnz = rowptr[M];
            __threadfence_system();  // the host reads out once the stream's event completes
            acc->sumsq = 0;
            acc->empty = 0;
            acc->maxlen = 0;
            acc->blocks_done = 0;
        }
    }
}

struct Entry {
    int device;
    const void *rowptr, *colidx;
    int64_t rows, cols;
    int64_t stats[5];
    bool pending;      // a re-measurement is in flight (its event not yet seen complete)
    cudaEvent_t ev;    // completion of the last measurement (its counters are in the host slot)
    StatsOut *h_stats;  // pinned host slot of this entry's counters, mapped for the device
    StatsOut *d_stats;  // the same slot's device address
    StatsAcc *acc;      // the pattern's device accumulators
};
constexpr int kCache = 64;
std::mutex g_mu;
Entry g_cache[kCache];
int g_used = 0, g_next = 0;
unsigned char *g_pinned = nullptr;  // kCache slots of 32 bytes (StatsOut), mapped into every device

bool same_key(const Entry &c, int dev, const gbsp_csr &A) {
    return c.device == dev && c.rowptr == A.rowptr && c.colidx == A.colidx && c.rows == A.rows && c.cols == A.cols;
}

// Enqueues one measurement of A's row lengths on s: one kernel, whose counters land in the
// entry's pinned slot; the entry's event marks their arrival.
int enqueue_measure(const gbsp_csr &A, cudaStream_t s, Entry &e) {
    int64_t blocks = (A.rows + 255) / 256;
    if (blocks > 4LL * sm_count()) blocks = 4LL * sm_count();
    if (blocks < 1) blocks = 1;
    row_stats_kernel<<<(unsigned)blocks, 256, 0, s>>>(A.rowptr, A.rows, e.acc, e.d_stats);
    count_launches(1);
    int st = check_launch("auto: row statistics");
    if (!st && cudaEventRecord(e.ev, s) != cudaSuccess) st = check_launch("auto: event");
    return st;
}

// Reads the entry's pinned slot into its statistics and decision.
void adopt(Entry &e) {
    e.stats[0] = e.rows;
    e.stats[1] = e.h_stats->nnz;
    e.stats[2] = (int64_t)e.h_stats->sumsq;
    e.stats[3] = (int64_t)e.h_stats->maxlen;
    e.stats[4] = (int64_t)e.h_stats->empty;
}

int rule(int op, const int64_t *st, int64_t b_bytes, int64_t row_bytes) {
    return op == kOpSddmm ? auto_sddmm_rule(st[0], st[1], st[2], st[3], b_bytes, row_bytes)
                          : auto_spmm_rule(st[0], st[1], st[2], st[3], b_bytes, row_bytes);
}

}  // namespace

// The split for a pattern with these row statistics (M rows, nnz entries, sum of squared
// lengths, longest row) and a dense operand of b_bytes bytes with rows of row_bytes:
// rows averaging under 12 entries with none past 128 take the row groups (several rows per
// warp); skewed rows (coefficient of variation above 1, or a longest row past 16 times the
// mean and past 256) take the merge path; even rows gathered from a B that overflows L2
// (more than 192 MB) in rows of at least 256 bytes also take the row groups, whose smaller
// register footprint keeps more CTAs, and so more gathers, in flight per SM while they wait
// on HBM (measured on 1,048,576^2 at 99.99%: 3.02 / 6.17 ms against 3.33 / 7.40 ms for the
// row split at N = 64 / 128); even rows of 128 bytes from a B past 96 MB take the merge path
// (same matrix, N = 32: 1.41 against 1.54 ms; on 65,536^2, where B sits in L2, the two are
// level); the rest the row split.
int auto_spmm_rule(int64_t M, int64_t nnz, int64_t sumsq, int64_t maxlen, int64_t b_bytes, int64_t row_bytes) {
    if (M <= 0 || nnz <= 0) return GBSP_VARIANT_ROWSPLIT;
    const double mean = (double)nnz / (double)M;
    const double var = (double)sumsq / (double)M - mean * mean;
    const double cv = var > 0 ? sqrt(var) / mean : 0.0;
    if (mean < 12.0 && maxlen <= 128) return GBSP_VARIANT_ROWGROUP;
    if (cv > 1.0 || (maxlen > 16.0 * mean && maxlen > 256)) return GBSP_VARIANT_MERGE;
    if (b_bytes > (192LL << 20) && row_bytes >= 256 && maxlen <= 4 * mean + 64) return GBSP_VARIANT_ROWGROUP;
    if (b_bytes > (96LL << 20) && row_bytes == 128 && maxlen <= 4 * mean + 64) return GBSP_VARIANT_MERGE;
    return GBSP_VARIANT_ROWSPLIT;
}

// The SDDMM split: rows averaging under 32 stored entries take the entry split (a row split
// would leave lanes idle); skewed rows (as for SpMM) the merge path; the rest the row split
// (with the paired FP32 layout it also leads on even rows whose Y overflows L2: 7.69 against
// 8.02 ms for the merge path on 1,048,576^2 at 99.99%, Kd = 128).  The operand size is
// accepted for the same signature as the SpMM rule.
int auto_sddmm_rule(int64_t M, int64_t nnz, int64_t sumsq, int64_t maxlen, int64_t, int64_t) {
    if (M <= 0 || nnz <= 0) return GBSP_VARIANT_ROWSPLIT;
    const double mean = (double)nnz / (double)M;
    const double var = (double)sumsq / (double)M - mean * mean;
    const double cv = var > 0 ? sqrt(var) / mean : 0.0;
    if (mean < 32.0) return GBSP_VARIANT_ENTRY;
    if (cv > 1.0 || (maxlen > 16.0 * mean && maxlen > 256)) return GBSP_VARIANT_MERGE;
    return GBSP_VARIANT_ROWSPLIT;
}

// The split AUTO takes for op (kOpSpmm, kOpSddmm) on A's pattern and the statistics behind it.  A pattern not seen
// before is measured at once (synchronising on the measurement's event).  A kept pattern
// uses its kept choice and queues a re-measurement on s; a later call adopts that
// measurement once its event has completed (queried, never waited for), so a different
// pattern that reuses the same addresses gets its own choice from then on.  Under stream
// capture nothing is queued: a kept choice is used, else the row split.
int auto_choice(const gbsp_csr &A, int op, int64_t b_bytes, int64_t row_bytes, cudaStream_t s, int *variant,
                int64_t *stats) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_launch("auto: current device");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return check_launch("auto: capture status");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lk(g_mu);
    int k = 0;
    while (k < g_used && !same_key(g_cache[k], dev, A)) ++k;
    const bool found = k < g_used;
    if (!found && (capturing || A.rows == 0)) {
        *variant = GBSP_VARIANT_ROWSPLIT;
        if (stats)
            for (int j = 0; j < 5; ++j) stats[j] = -1;
        return GBSP_OK;
    }
    int st = GBSP_OK;
    if (found) {
        Entry &e = g_cache[k];
        if (e.pending) {
            const cudaError_t q = cudaEventQuery(e.ev);
            if (q == cudaSuccess) {
                adopt(e);
                e.pending = false;
            } else if (q == cudaErrorNotReady) {
                if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
            } else {
                return check_launch("auto: measurement");
            }
        }
        *variant = rule(op, e.stats, b_bytes, row_bytes);
        if (stats)
            for (int j = 0; j < 5; ++j) stats[j] = e.stats[j];
        if (!capturing && !e.pending && !(st = enqueue_measure(A, s, e))) e.pending = true;
        return st;
    }
    // a new pattern: take a slot (the oldest when all are used) and measure now
    if (!g_pinned) {
        if (cudaHostAlloc(&g_pinned, (size_t)kCache * 32, cudaHostAllocPortable | cudaHostAllocMapped) !=
            cudaSuccess) {
            g_pinned = nullptr;
            cudaGetLastError();
            return fail(GBSP_ERR_OOM, "auto: pinned host slots could not be allocated");
        }
    }
    const int slot = g_next;
    Entry &e = g_cache[slot];
    if (slot < g_used && e.ev) {
        if (e.pending) cudaEventSynchronize(e.ev);  // its kernel writes the slot being reused
        cudaEventDestroy(e.ev);
        cudaFree(e.acc);
    }
    e = Entry{};
    if (cudaEventCreateWithFlags(&e.ev, cudaEventDisableTiming) != cudaSuccess) {
        e.ev = nullptr;
        return check_launch("auto: event");
    }
    e.device = dev;
    e.rowptr = A.rowptr;
    e.colidx = A.colidx;
    e.rows = A.rows;
    e.cols = A.cols;
    e.h_stats = reinterpret_cast<StatsOut *>(g_pinned + 32 * slot);
    void *dslot = nullptr;
    if (cudaHostGetDevicePointer(&dslot, e.h_stats, 0) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&e.acc), sizeof(StatsAcc)) != cudaSuccess ||
        cudaMemsetAsync(e.acc, 0, sizeof(StatsAcc), s) != cudaSuccess) {
        st = check_launch("auto: counters");
        cudaFree(e.acc);
        cudaEventDestroy(e.ev);
        e = Entry{};
        return st ? st : fail(GBSP_ERR_CUDA, "auto: counters");
    }
    e.d_stats = static_cast<StatsOut *>(dslot);
    if ((st = enqueue_measure(A, s, e)) || cudaEventSynchronize(e.ev) != cudaSuccess) {
        if (!st) st = check_launch("auto: measurement");
        cudaFree(e.acc);
        cudaEventDestroy(e.ev);
        e = Entry{};
        return st;
    }
    adopt(e);
    g_next = (g_next + 1) % kCache;
    if (g_used < kCache) ++g_used;
    *variant = rule(op, e.stats, b_bytes, row_bytes);
    if (stats)
        for (int j = 0; j < 5; ++j) stats[j] = e.stats[j];
    return GBSP_OK;
}

void auto_forget_all() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < g_used; ++k) {
        if (g_cache[k].ev) {
            if (g_cache[k].pending) cudaEventSynchronize(g_cache[k].ev);
            cudaEventDestroy(g_cache[k].ev);
        }
        cudaFree(g_cache[k].acc);
        g_cache[k] = Entry{};
    }
    g_used = 0;
    g_next = 0;
}

}  // namespace gbsp

using namespace gbsp;

GBSP_EXPORT int gbsp_auto_choice(const gbsp_csr *A, int32_t op, int64_t b_bytes, int64_t row_bytes, void *stream,
                                 int32_t *variant, int64_t *stats) {
    if (!A || !variant) return fail(GBSP_ERR_INVALID_ARG, "auto choice: null argument");
    if (op != kOpSpmm && op != kOpSddmm) return fail(GBSP_ERR_INVALID_ARG, "auto choice: op must be 0 or 1");
    if (A->rows < 0 || A->rows > 2147483647LL || A->cols < 0 || (A->rows > 0 && !A->rowptr))
        return fail(GBSP_ERR_INVALID_ARG, "auto choice: bad CSR");
    int v = GBSP_VARIANT_ROWSPLIT;
    const int st = auto_choice(*A, op, b_bytes, row_bytes, static_cast<cudaStream_t>(stream), &v, stats);
    if (st) return st;
    *variant = v;
    return ok();
}

GBSP_EXPORT void gbsp_auto_forget(void) { auto_forget_all(); }

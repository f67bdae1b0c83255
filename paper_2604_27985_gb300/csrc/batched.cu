// Grouped SpMM and SDDMM over many problems of uneven size in one persistent launch.
//
// The work list holds tiles of consecutive rows of one problem with about 512 stored
// entries each, grouped by the lane layout their problem's width needs (one class per
// layout).  Each class runs as one persistent launch whose warps take tiles from the class's
// atomic ticket and run the row kernels of spmm_kernels.cuh / sddmm_kernels.cuh on them (for
// SDDMM tiles of short rows, the entry split).  One kernel per layout keeps each launch's
// registers to what its layout needs (a single kernel holding every layout needed 255 and
// spilled).  The ticket resets and the launches are recorded once into a CUDA graph;
// executing a plan replays it.
#include <vector>

#include "sddmm_kernels.cuh"
#include "spmm_kernels.cuh"

namespace gbsp {
namespace batched {

struct Tile {
    int32_t problem, row0, row1;
};

enum Kind { kSpmm = 0, kSddmm = 1 };

struct GroupArgs {
    const SpmmProblem *spmm;
    const SddmmProblem *sddmm;
    const Tile *tiles;  // this class's tiles
    int ntiles;
    unsigned *ticket;   // this class's ticket
};

constexpr int kClasses = 5;

// Lane-layout class of a problem from its vectors per dense row: SpMM 0: <= 8 (8 lanes x 1),
// 1: <= 16 (8 x 2), 2: wider (16 x 2 per 32-vector column tile); SDDMM 0: <= 4 (4 x 1),
// 1: <= 8 (8 x 1), 2: <= 16 (8 x 2), 3: <= 32 (16 x 2), 4: <= 64 (32 x 2).
int layout_class(int kind, int nvec) {
    if (kind == kSpmm) return nvec <= 8 ? 0 : nvec <= 16 ? 1 : 2;
    return nvec <= 4 ? 0 : nvec <= 8 ? 1 : nvec <= 16 ? 2 : nvec <= 32 ? 3 : 4;
}

template <class EL, int LPN, int VPL, int U>
__device__ __forceinline__ void spmm_rows(const SpmmProblem &P, int r0, int r1, int lane) {
    using namespace spmm_detail;
    constexpr int TW = LPN * VPL * EL::V;
    for (int tile = 0; tile * TW < P.N; ++tile) {
        const int col_base = tile * TW + (lane % LPN) * EL::V;
        const bool full = (tile + 1) * TW <= P.N;
        for (int row = r0; row < r1; ++row) {
            float acc[VPL][EL::V];
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int k = 0; k < EL::V; ++k) acc[v][k] = 0.f;
            const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
            if (full)
                gather_range<EL, LPN, VPL, U, false>(P, p0, p1, acc, lane, col_base);
            else
                gather_range<EL, LPN, VPL, U, true>(P, p0, p1, acc, lane, col_base);
            reduce_groups<EL, LPN, VPL>(acc);
            store_row<EL, LPN, VPL>(P.C + (int64_t)row * P.ldc, acc, lane, col_base, P.N, 1.0f);
        }
    }
}

template <class EL, int LPN, int VPL>
__device__ __forceinline__ void sddmm_rows(const SddmmProblem &P, int r0, int r1, int lane) {
    using namespace sddmm_detail;
    const bool full = P.Kd == LPN * VPL * EL::V;
    const int64_t e0 = __ldg(P.rowptr + r0), e1 = __ldg(P.rowptr + r1);
    if (e1 - e0 < 32 * (int64_t)(r1 - r0)) {  // short rows: the tile's entries 32 at a time across rows
        if (e1 > e0) {
            if (full)
                sddmm_entries<EL, LPN, VPL, false>(P, e0, e1, r0, lane);
            else
                sddmm_entries<EL, LPN, VPL, true>(P, e0, e1, r0, lane);
        }
        return;
    }
    for (int row = r0; row < r1; ++row) {
        const int64_t p0 = __ldg(P.rowptr + row), p1 = __ldg(P.rowptr + row + 1);
        if (p0 == p1) continue;
        if (full)
            sddmm_segment<EL, LPN, VPL, false>(P, row, p0, p1, lane);
        else
            sddmm_segment<EL, LPN, VPL, true>(P, row, p0, p1, lane);
    }
}

template <class EL, int KIND, int CLASS>
__device__ __forceinline__ void run_tile(const GroupArgs &a, const Tile &t, int lane) {
    if constexpr (KIND == kSpmm) {
        const SpmmProblem &P = a.spmm[t.problem];
        if constexpr (CLASS == 0) spmm_rows<EL, 8, 1, 8>(P, t.row0, t.row1, lane);
        else if constexpr (CLASS == 1) spmm_rows<EL, 8, 2, 4>(P, t.row0, t.row1, lane);
        else spmm_rows<EL, 16, 2, 4>(P, t.row0, t.row1, lane);  // 32 vectors per column tile
    } else {
        const SddmmProblem &P = a.sddmm[t.problem];
        if constexpr (CLASS == 0) sddmm_rows<EL, 4, 1>(P, t.row0, t.row1, lane);
        else if constexpr (CLASS == 1) sddmm_rows<EL, 8, 1>(P, t.row0, t.row1, lane);
        else if constexpr (CLASS == 2) sddmm_rows<EL, 8, 2>(P, t.row0, t.row1, lane);
        else if constexpr (CLASS == 3) sddmm_rows<EL, 16, 2>(P, t.row0, t.row1, lane);
        else sddmm_rows<EL, 32, 2>(P, t.row0, t.row1, lane);
    }
}

template <class EL, int KIND, int CLASS>
__global__ void __launch_bounds__(256) grouped_kernel(const GroupArgs a) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= (unsigned)a.ntiles) return;
        run_tile<EL, KIND, CLASS>(a, a.tiles[t], lane);
    }
}

}  // namespace batched
}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::batched;

struct gbsp_batch_plan {
    int kind, dtype, G, ntiles;
    int class_begin[kClasses + 1];  // tiles of layout class c: [class_begin[c], class_begin[c + 1])
    int launches;
    int64_t nnz;
    SpmmProblem *d_spmm;
    SddmmProblem *d_sddmm;
    Tile *d_tiles;
    unsigned *d_ticket;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

void batch_free(gbsp_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_spmm);
    cudaFree(p->d_sddmm);
    cudaFree(p->d_tiles);
    cudaFree(p->d_ticket);
    delete p;
}

int elem_bytes(int dt) { return dt == GBSP_F32 ? 4 : dt == GBSP_BF16 ? 2 : 0; }

// Tiles of consecutive rows with about 512 entries (at most 256 rows), from the host copy
// of a problem's row pointers.
int add_tiles(const gbsp_csr &A, int g, cudaStream_t s, std::vector<Tile> &tiles, int64_t &nnz) {
    std::vector<int32_t> rp((size_t)A.rows + 1);
    if (A.rows > 0 &&
        (cudaMemcpyAsync(rp.data(), A.rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        return check_launch("batch plan rowptr copy");
    if (A.rows > 0 && (rp[0] != 0 || (int64_t)rp[A.rows] != A.nnz))
        return fail(GBSP_ERR_INVALID_CSR, "batch plan: problem %d: rowptr[0] != 0 or rowptr[rows] != nnz", g);
    int32_t r0 = 0;
    while (r0 < A.rows) {
        int32_t r1 = r0 + 1;
        while (r1 < A.rows && rp[r1 + 1] - rp[r0] <= 512 && r1 - r0 < 256) ++r1;
        tiles.push_back(Tile{g, r0, r1});
        r0 = r1;
    }
    nnz += A.nnz;
    return GBSP_OK;
}

template <class EL, int KIND, int CLASS>
void launch_class(gbsp_batch_plan *p, cudaStream_t cap) {
    const int b = p->class_begin[CLASS], n = p->class_begin[CLASS + 1] - b;
    if (n <= 0) return;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_kernel<EL, KIND, CLASS>, 256, 0);
    int nblocks = sm_count() * (per_sm < 1 ? 1 : per_sm);
    if (nblocks > (n + 7) / 8) nblocks = (n + 7) / 8;  // no more warps than tiles
    GroupArgs args{p->d_spmm, p->d_sddmm, p->d_tiles + b, n, p->d_ticket + CLASS};
    grouped_kernel<EL, KIND, CLASS><<<nblocks, 256, 0, cap>>>(args);
    ++p->launches;
}

template <class EL, int KIND>
int record(gbsp_batch_plan *p) {
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return check_launch("batch stream");
    bool okc = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    p->launches = 0;
    if (okc) {
        cudaMemsetAsync(p->d_ticket, 0, sizeof(unsigned) * kClasses, cap);
        launch_class<EL, KIND, 0>(p, cap);
        launch_class<EL, KIND, 1>(p, cap);
        launch_class<EL, KIND, 2>(p, cap);
        if constexpr (KIND == kSddmm) {
            launch_class<EL, KIND, 3>(p, cap);
            launch_class<EL, KIND, 4>(p, cap);
        }
        okc = cudaStreamEndCapture(cap, &p->graph) == cudaSuccess;
    }
    okc = okc && cudaGraphInstantiate(&p->exec, p->graph, 0) == cudaSuccess;
    cudaStreamDestroy(cap);
    if (!okc) {
        int st = check_launch("batch capture");
        return st ? st : fail(GBSP_ERR_CUDA, "batch plan: graph capture failed");
    }
    return GBSP_OK;
}

int create(int kind, int G, const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, const gbsp_dense *X,
           const gbsp_dense *Y, float *const *out, void *stream, gbsp_batch_plan **res) {
    if (!res) return fail(GBSP_ERR_INVALID_ARG, "batch plan: null output");
    *res = nullptr;
    if (G < 0 || (G > 0 && (!A || (kind == kSpmm ? (!B || !C) : (!X || !Y || !out)))))
        return fail(GBSP_ERR_INVALID_ARG, "batch plan: bad arrays");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<SpmmProblem> sp;
    std::vector<SddmmProblem> sd;
    std::vector<Tile> by_class[kClasses];
    int64_t nnz = 0;
    const int dtype = kind == kSpmm ? (G > 0 ? B[0].dtype : GBSP_F32) : (G > 0 ? X[0].dtype : GBSP_F32);
    const int eb = elem_bytes(dtype);
    if (eb == 0) return fail(GBSP_ERR_UNSUPPORTED, "batch plan: FP32 or BF16 dense operands");
    const int V = 16 / eb;
    for (int g = 0; g < G; ++g) {
        const gbsp_csr &a = A[g];
        if (a.rows < 0 || a.cols < 0 || a.rows > 2147483647LL || a.cols > 2147483647LL || a.nnz < 0 ||
            (a.rows > 0 && !a.rowptr) || (a.nnz > 0 && (!a.colidx || !a.vals)))
            return fail(GBSP_ERR_INVALID_ARG, "batch plan: problem %d: bad CSR", g);
        if (kind == kSpmm) {
            const gbsp_dense &b = B[g], &c = C[g];
            if (a.dtype != dtype || b.dtype != dtype || c.dtype != GBSP_F32 || b.rows != a.cols || c.rows != a.rows ||
                c.cols != b.cols || b.ld < b.cols || c.ld < c.cols)
                return fail(GBSP_ERR_INVALID_ARG, "batch plan: problem %d: shapes or dtypes", g);
            if (b.cols % V || b.ld % V || c.ld % 4 || !aligned16(b.data) || !aligned16(c.data))
                return fail(GBSP_ERR_ALIGN, "batch plan: problem %d: widths and ld multiples of %d, 16-byte aligned",
                            g, V);
            SpmmProblem p{};
            p.M = (int32_t)a.rows;
            p.K = (int32_t)a.cols;
            p.N = (int32_t)b.cols;
            p.nnz = a.nnz;
            p.rowptr = a.rowptr;
            p.colidx = a.colidx;
            p.vals = a.vals;
            p.B = b.data;
            p.ldb = b.ld;
            p.C = static_cast<float *>(c.data);
            p.ldc = c.ld;
            p.dtype = dtype;
            sp.push_back(p);
        } else {
            const gbsp_dense &x = X[g], &y = Y[g];
            if (a.dtype != GBSP_F32 || x.dtype != dtype || y.dtype != dtype || x.rows != a.rows || y.rows != a.cols ||
                x.cols != y.cols || x.ld < x.cols || y.ld < y.cols || (a.nnz > 0 && !out[g]))
                return fail(GBSP_ERR_INVALID_ARG, "batch plan: problem %d: shapes or dtypes", g);
            if (x.cols % V || x.ld % V || y.ld % V || x.cols > 64 * V || !aligned16(x.data) || !aligned16(y.data))
                return fail(GBSP_ERR_ALIGN, "batch plan: problem %d: Kd and ld multiples of %d, Kd <= %d, aligned",
                            g, V, 64 * V);
            SddmmProblem p{};
            p.M = (int32_t)a.rows;
            p.N = (int32_t)a.cols;
            p.Kd = (int32_t)x.cols;
            p.nnz = a.nnz;
            p.rowptr = a.rowptr;
            p.colidx = a.colidx;
            p.svals = static_cast<const float *>(a.vals);
            p.X = x.data;
            p.ldx = x.ld;
            p.Y = y.data;
            p.ldy = y.ld;
            p.out = out[g];
            p.dtype = dtype;
            sd.push_back(p);
        }
        const int nvec = (int)((kind == kSpmm ? B[g].cols : X[g].cols) / V);
        int st = add_tiles(a, g, s, by_class[layout_class(kind, nvec)], nnz);
        if (st) return st;
    }
    std::vector<Tile> tiles;
    int class_begin[kClasses + 1];
    for (int c = 0; c < kClasses; ++c) {
        class_begin[c] = (int)tiles.size();
        tiles.insert(tiles.end(), by_class[c].begin(), by_class[c].end());
    }
    class_begin[kClasses] = (int)tiles.size();
    gbsp_batch_plan *p = new gbsp_batch_plan();
    p->kind = kind;
    p->dtype = dtype;
    p->G = G;
    p->ntiles = (int)tiles.size();
    for (int c = 0; c <= kClasses; ++c) p->class_begin[c] = class_begin[c];
    p->nnz = nnz;
    const size_t nsp = sp.size(), nsd = sd.size();
    if (cudaMalloc(&p->d_spmm, sizeof(SpmmProblem) * (nsp ? nsp : 1)) != cudaSuccess ||
        cudaMalloc(&p->d_sddmm, sizeof(SddmmProblem) * (nsd ? nsd : 1)) != cudaSuccess ||
        cudaMalloc(&p->d_tiles, sizeof(Tile) * (tiles.empty() ? 1 : tiles.size())) != cudaSuccess ||
        cudaMalloc(&p->d_ticket, sizeof(unsigned) * kClasses) != cudaSuccess) {
        cudaGetLastError();
        batch_free(p);
        return fail(GBSP_ERR_OOM, "batch plan: allocation failed");
    }
    // stream-ordered uploads, complete before the host vectors go out of scope and before
    // the graph that reads them is recorded or replayed
    if ((nsp && cudaMemcpyAsync(p->d_spmm, sp.data(), sizeof(SpmmProblem) * nsp, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess) ||
        (nsd && cudaMemcpyAsync(p->d_sddmm, sd.data(), sizeof(SddmmProblem) * nsd, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess) ||
        (!tiles.empty() && cudaMemcpyAsync(p->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(),
                                           cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        int st = check_launch("batch plan upload");
        batch_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "batch plan upload");
    }
    int st;
    if (kind == kSpmm)
        st = dtype == GBSP_F32 ? record<F32, kSpmm>(p) : record<BF16, kSpmm>(p);
    else
        st = dtype == GBSP_F32 ? record<F32, kSddmm>(p) : record<BF16, kSddmm>(p);
    if (st) {
        batch_free(p);
        return st;
    }
    *res = p;
    return GBSP_OK;
}

}  // namespace

GBSP_EXPORT int gbsp_batch_plan_create_spmm(int G, const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C,
                                            void *stream, gbsp_batch_plan **out) {
    int st = create(kSpmm, G, A, B, C, nullptr, nullptr, nullptr, stream, out);
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_batch_plan_create_sddmm(int G, const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y,
                                             float *const *out, void *stream, gbsp_batch_plan **res) {
    int st = create(kSddmm, G, S, nullptr, nullptr, X, Y, out, stream, res);
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_batch_plan_execute(const gbsp_batch_plan *p, void *stream) {
    if (!p) return fail(GBSP_ERR_INVALID_ARG, "batch execute: null plan");
    if (cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return check_launch("batch execute");
    count_launches(p->launches);
    return ok();
}

GBSP_EXPORT void gbsp_batch_plan_destroy(gbsp_batch_plan *p) { batch_free(p); }

GBSP_EXPORT int spmm_csr_batched(int G, const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, void *stream) {
    gbsp_batch_plan *p = nullptr;
    int st = create(kSpmm, G, A, B, C, nullptr, nullptr, nullptr, stream, &p);
    if (st) return st;
    st = gbsp_batch_plan_execute(p, stream);
    if (!st && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) st = check_launch("batched");
    batch_free(p);
    return st ? st : ok();
}

GBSP_EXPORT int sddmm_csr_batched(int G, const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y,
                                  float *const *out, void *stream) {
    gbsp_batch_plan *p = nullptr;
    int st = create(kSddmm, G, S, nullptr, nullptr, X, Y, out, stream, &p);
    if (st) return st;
    st = gbsp_batch_plan_execute(p, stream);
    if (!st && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) st = check_launch("batched");
    batch_free(p);
    return st ? st : ok();
}

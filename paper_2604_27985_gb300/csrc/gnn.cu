// Batched graph chain: for each graph g of a batch,
//   E_g = S_g o (H_g H_g^T)   on the pattern of S_g   (SDDMM, Eq. 2 with X = Y = H_g)
//   O_g = E_g H_g                                       (SpMM, Eq. 1 with A's values E_g)
// with BF16 features H_g (n_g x N_g, N_g a multiple of 8 up to 256), FP32 E_g and
// accumulation, BF16 O_g (round to nearest even).
//
// One persistent launch covers the whole batch: the work list holds tiles of consecutive
// rows (at most 63) of one graph with about the same number of edges (512 by default, so
// the tiles in flight at once span few graphs and their features stay in L2); warps take
// tiles from an atomic ticket in graph order.  Each row is fused: every gathered H_j serves both the dot product with H_i (its
// edge's E value, reduced across the lane group by an xor butterfly) and the accumulation
// E_ij * H_j into O_i, so H_j is read once per edge.  The launch (and the ticket reset) is
// recorded once into a CUDA graph and replayed per execution.
//
// The GAT-style form (GBSP_GNN_SOFTMAX) puts a softmax over each row's scores between the
// two products: alpha_ij = exp(E_ij - max_k E_ik) / sum_k exp(E_ik - max_k E_ik), O_i =
// sum_j alpha_ij H_j, and E receives alpha.  It keeps the single gather per edge with an
// online softmax: each lane group folds its edges into a running sum and accumulator
// against a reference score, and the groups' states are merged at the row's end.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gbsp {
namespace gnn {

struct GraphDesc {
    const int32_t *rowptr;  // n + 1
    const int32_t *colidx;  // local column indices
    const float *svals;
    const uint16_t *H;  // BF16 n x N, leading dimension ldh
    uint16_t *O;        // BF16 n x N, leading dimension ldo
    float *E;           // nnz
    int64_t ldh, ldo;
    int32_t n, N;
};

struct Tile {
    int32_t graph, row0, row1;
};

struct GnnArgs {
    const GraphDesc *graphs;
    const Tile *tiles;
    int ntiles;
    unsigned *ticket;
};

// One group step: U edges per lane group (entries q + u * G + sub of the current chunk):
// gather H_j, dot with H_i across the group (xor butterfly), E_ij = s_ij * dot (stored by
// the group's first lane), then E_ij * H_j into the accumulator.
template <int LPN, int VPL, int U>
__device__ __forceinline__ void gnn_step(const uint4 *Hv, int64_t ldv, const bool (&colok)[VPL], int c, float s,
                                         int q, int cnt, int sub, int sl, const float (&x)[VPL][8],
                                         float (&acc)[VPL][8], float *E, int64_t base) {
    constexpr int G = 32 / LPN;
    uint4 raw[U][VPL];
    float sj[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = q + u * G + sub;
        const int cj = __shfl_sync(FULL, c, idx & 31);
        sj[u] = __shfl_sync(FULL, s, idx & 31);
        ok[u] = idx < cnt;
        const uint4 *rp = Hv + (int64_t)cj * ldv;
#pragma unroll
        for (int v = 0; v < VPL; ++v) raw[u][v] = (ok[u] && colok[v]) ? __ldg(rp + v * LPN) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        float f[VPL][8];
        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            BF16::unpack(raw[u][v], f[v]);
            dot2(x[v], f[v], d2);
        }
        float dot = d2.x + d2.y;
#pragma unroll
        for (int off = LPN / 2; off >= 1; off >>= 1) dot += __shfl_xor_sync(FULL, dot, off);
        const float e = sj[u] * dot;
        if (sl == 0 && ok[u]) __stcs(E + base + q + u * G + sub, e);  // written once: evict first, keep H in L2
#pragma unroll
        for (int v = 0; v < VPL; ++v) axpy2(e, f[v], acc[v]);
    }
}

// The softmax form of a group step (the GAT-style chain).  Scores are kept in base-2 units,
// z = e log2(e), so that every weight is one exp2f.  Each edge is folded in as soon as its
// score is known, against the group's reference m: acc += 2^(z - m) H_j, l += 2^(z - m).
// m is the first score of the row and moves up (rescaling acc and l by 2^(m - m')) only when
// a score exceeds it by more than kLazy, so weights stay below 2^kLazy and the rescale is
// rare; softmax does not depend on the reference, so the result is the same.  Lane L also
// collects, by one shuffle per edge, the score of the chunk's entry L.
constexpr float kLazy = 12.f;

template <int LPN, int VPL, int U>
__device__ __forceinline__ void gnn_step_softmax(const uint4 *Hv, int64_t ldv, const bool (&colok)[VPL], int c,
                                                 float s, int q, int cnt, int sub, int lane,
                                                 const float (&x)[VPL][8], float (&acc)[VPL][8], float &m, float &l,
                                                 float &mine) {
    constexpr int G = 32 / LPN;
    uint4 raw[U][VPL];
    float sj[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = q + u * G + sub;
        const int cj = __shfl_sync(FULL, c, idx & 31);
        sj[u] = __shfl_sync(FULL, s, idx & 31);
        ok[u] = idx < cnt;
        const uint4 *rp = Hv + (int64_t)cj * ldv;
#pragma unroll
        for (int v = 0; v < VPL; ++v) raw[u][v] = (ok[u] && colok[v]) ? __ldg(rp + v * LPN) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        float f[VPL][8];
        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            BF16::unpack(raw[u][v], f[v]);
            dot2(x[v], f[v], d2);
        }
        float dot = d2.x + d2.y;
#pragma unroll
        for (int off = LPN / 2; off >= 1; off >>= 1) dot += __shfl_xor_sync(FULL, dot, off);
        const float z = sj[u] * dot * 1.4426950408889634f;
        const int rel = lane - (q + u * G);  // the chunk entry this lane collects, if in this step
        const float zg = __shfl_sync(FULL, z, (rel & (G - 1)) * LPN);
        if (rel >= 0 && rel < G) mine = zg;
        if (!ok[u]) continue;
        if (z > m + kLazy) {  // also the row's first edge, while m is -inf
            const float r = exp2f(m - z);
            l *= r;
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[v][t] *= r;
            m = z;
        }
        const float w = exp2f(z - m);
        l += w;
#pragma unroll
        for (int v = 0; v < VPL; ++v) axpy2(w, f[v], acc[v]);
    }
}

// The rows [r0, r1) (at most 63) of one graph, one after another, with LPN lanes per edge
// and VPL 16-byte BF16 vectors (8 features each) per lane.  The tile's row pointers sit in
// two registers per lane; the next row's first 32 column indices and values and its H row
// are loaded while the current row computes.  Full steps take U edges per group; the rest
// of a chunk goes one edge per group, so a row with a single edge costs one step.
template <int LPN, int VPL, int U, bool SOFTMAX>
__device__ __forceinline__ void gnn_tile(const GraphDesc &g, int r0, int r1, int lane) {
    constexpr int G = 32 / LPN;
    constexpr int STEP = G * U;
    static_assert(STEP <= 32 && 32 % STEP == 0, "whole steps per chunk");
    const int sl = lane % LPN, sub = lane / LPN;
    bool colok[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) colok[v] = (v * LPN + sl) * 8 < g.N;
    const uint4 *Hv = reinterpret_cast<const uint4 *>(g.H) + sl;
    const int64_t ldv = g.ldh / 8;
    const int nrows = r1 - r0;
    const int rp_a = lane <= nrows ? g.rowptr[r0 + lane] : 0;
    const int rp_b = lane + 32 <= nrows ? g.rowptr[r0 + 32 + lane] : 0;
    auto start = [&](int k) {
        const int a = __shfl_sync(FULL, rp_a, k & 31), b = __shfl_sync(FULL, rp_b, k & 31);
        return k < 32 ? a : b;
    };
    int64_t p0 = start(0), p1 = start(1);
    int c = 0;
    float s = 0.f;
    if (p0 + lane < p1) {
        c = ld_stream(g.colidx + p0 + lane);
        s = ld_stream(g.svals + p0 + lane);
    }
    uint4 xraw[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) xraw[v] = colok[v] ? __ldg(Hv + (int64_t)r0 * ldv + v * LPN) : make_uint4(0, 0, 0, 0);
    for (int k = 0; k < nrows; ++k) {
        const int row = r0 + k;
        // next row, loaded now
        int64_t q1 = p1;
        int cn = 0;
        float sn = 0.f;
        uint4 xn[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) xn[v] = make_uint4(0, 0, 0, 0);
        if (k + 1 < nrows) {
            q1 = start(k + 2);
            if (p1 + lane < q1) {
                cn = ld_stream(g.colidx + p1 + lane);
                sn = ld_stream(g.svals + p1 + lane);
            }
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                if (colok[v]) xn[v] = __ldg(Hv + (int64_t)(row + 1) * ldv + v * LPN);
        }
        float x[VPL][8], acc[VPL][8];
        float m = -INFINITY, l = 0.f, mine = 0.f;  // softmax: the group's reference and sum; this lane's score
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            BF16::unpack(xraw[v], x[v]);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc[v][t] = 0.f;
        }
        for (int64_t base = p0; base < p1; base += 32) {
            if (base > p0) {  // rows longer than 32 edges load their later chunks here
                c = 0;
                s = 0.f;
                if (base + lane < p1) {
                    c = ld_stream(g.colidx + base + lane);
                    s = ld_stream(g.svals + base + lane);
                }
            }
            const int cnt = (int)min((int64_t)32, p1 - base);
            int q = 0;
            if constexpr (SOFTMAX) {
#pragma unroll 1
                for (; q + STEP <= cnt; q += STEP)
                    gnn_step_softmax<LPN, VPL, U>(Hv, ldv, colok, c, s, q, cnt, sub, lane, x, acc, m, l, mine);
#pragma unroll 1
                for (; q < cnt; q += G)
                    gnn_step_softmax<LPN, VPL, 1>(Hv, ldv, colok, c, s, q, cnt, sub, lane, x, acc, m, l, mine);
                if (base + 32 < p1) g.E[base + lane] = mine;  // a later chunk follows: park the scores in E
            } else {
#pragma unroll 1
                for (; q + STEP <= cnt; q += STEP)
                    gnn_step<LPN, VPL, U>(Hv, ldv, colok, c, s, q, cnt, sub, sl, x, acc, g.E, base);
#pragma unroll 1
                for (; q < cnt; q += G)
                    gnn_step<LPN, VPL, 1>(Hv, ldv, colok, c, s, q, cnt, sub, sl, x, acc, g.E, base);
            }
        }
        float row_max = 0.f, inv_sum = 0.f;
        if constexpr (SOFTMAX) {  // the groups' states merged: one maximum, rescaled sums
            row_max = m;
#pragma unroll
            for (int off = LPN; off < 32; off <<= 1) row_max = fmaxf(row_max, __shfl_xor_sync(FULL, row_max, off));
            const float f = m == -INFINITY ? 0.f : exp2f(m - row_max);
            l *= f;
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[v][t] *= f;
#pragma unroll
            for (int off = LPN; off < 32; off <<= 1) l += __shfl_xor_sync(FULL, l, off);
            inv_sum = l > 0.f ? 1.0f / l : 0.f;
        }
#pragma unroll
        for (int off = LPN; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[v][t] += __shfl_xor_sync(FULL, acc[v][t], off);
        if constexpr (SOFTMAX) {
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[v][t] *= inv_sum;
            // the weights: the last chunk's scores are in registers, earlier chunks' in E (each
            // lane reads back what it stored)
            const int64_t last = p1 > p0 ? p0 + ((p1 - p0 - 1) & ~(int64_t)31) : p0;  // the last chunk's start
            int64_t p = p0 + lane;
            // plain stores here: evict-first ones measured 8.61 against 7.38 ms on the 512 graphs
            for (; p < last; p += 32) g.E[p] = exp2f(g.E[p] - row_max) * inv_sum;
            if (p < p1) g.E[p] = exp2f(mine - row_max) * inv_sum;
        }
        if (lane < LPN) {
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                if (!colok[v]) continue;
                uint32_t w[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(acc[v][2 * t], acc[v][2 * t + 1]);
                    w[t] = *reinterpret_cast<uint32_t *>(&h);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(g.O + (int64_t)row * g.ldo) + v * LPN + sl;
                if constexpr (SOFTMAX)
                    *dst = make_uint4(w[0], w[1], w[2], w[3]);
                else
                    __stcs(dst, make_uint4(w[0], w[1], w[2], w[3]));  // written once: evict first, keep H in L2
            }
        }
        p0 = p1;
        p1 = q1;
        c = cn;
        s = sn;
#pragma unroll
        for (int v = 0; v < VPL; ++v) xraw[v] = xn[v];
    }
}

template <bool SOFTMAX>
__global__ void __launch_bounds__(256, 3) gnn_kernel(const GnnArgs a) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= (unsigned)a.ntiles) return;
        const Tile tile = a.tiles[t];
        const GraphDesc g = a.graphs[tile.graph];
        // The softmax form takes fewer edges per group step (2 and 1 instead of 4 and 2): its
        // steps hold more live state, and this keeps it at three CTAs per SM without spills.
        if (g.N <= 64)
            gnn_tile<8, 1, SOFTMAX ? 2 : 4, SOFTMAX>(g, tile.row0, tile.row1, lane);
        else if (g.N <= 128)
            gnn_tile<8, 2, SOFTMAX ? 1 : 2, SOFTMAX>(g, tile.row0, tile.row1, lane);
        else
            gnn_tile<16, 2, SOFTMAX ? 1 : 2, SOFTMAX>(g, tile.row0, tile.row1, lane);
    }
}

}  // namespace gnn
}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::gnn;

struct gbsp_gnn_plan {
    int device;
    int G;
    int ntiles;
    int64_t nnz, rows;
    GraphDesc *d_graphs;
    Tile *d_tiles;
    unsigned *d_ticket;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

void gnn_free(gbsp_gnn_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_graphs);
    cudaFree(p->d_tiles);
    cudaFree(p->d_ticket);
    delete p;
}

}  // namespace

GBSP_EXPORT int gbsp_gnn_plan_create_ex(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E,
                                        gbsp_dense *O, int32_t edges_per_tile, int32_t flags, void *stream,
                                        gbsp_gnn_plan **out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "gnn plan: null output");
    *out = nullptr;
    if (flags & ~GBSP_GNN_SOFTMAX) return fail(GBSP_ERR_INVALID_ARG, "gnn plan: unknown flags %d", flags);
    const bool softmax = (flags & GBSP_GNN_SOFTMAX) != 0;
    if (G < 0 || (G > 0 && (!S || !H || !E || !O))) return fail(GBSP_ERR_INVALID_ARG, "gnn plan: bad arrays");
    if (edges_per_tile <= 0) edges_per_tile = 512;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<GraphDesc> graphs(G);
    std::vector<Tile> tiles;
    std::vector<int32_t> rp;
    int64_t nnz = 0, rows = 0;
    for (int g = 0; g < G; ++g) {
        const gbsp_csr &a = S[g];
        const gbsp_dense &h = H[g], &o = O[g];
        if (a.rows != a.cols || a.rows < 0 || a.rows > 2147483647LL || a.nnz < 0 || a.dtype != GBSP_F32 ||
            (a.rows > 0 && !a.rowptr) || (a.nnz > 0 && (!a.colidx || !a.vals || !E[g])))
            return fail(GBSP_ERR_INVALID_ARG, "gnn plan: graph %d: S must be a square FP32 CSR with nnz given", g);
        if (h.dtype != GBSP_BF16 || o.dtype != GBSP_BF16 || h.rows != a.rows || o.rows != a.rows ||
            h.cols != o.cols || h.ld < h.cols || o.ld < o.cols)
            return fail(GBSP_ERR_INVALID_ARG, "gnn plan: graph %d: H and O must be BF16 n x N", g);
        if (h.cols % 8 || h.cols > 256 || h.ld % 8 || o.ld % 8 || !aligned16(h.data) || !aligned16(o.data))
            return fail(GBSP_ERR_UNSUPPORTED, "gnn plan: graph %d: N must be a multiple of 8 up to 256 with "
                        "16-byte aligned rows", g);
        graphs[g] = GraphDesc{a.rowptr, a.colidx, static_cast<const float *>(a.vals),
                              static_cast<const uint16_t *>(h.data), static_cast<uint16_t *>(o.data), E[g],
                              h.ld, o.ld, (int32_t)a.rows, (int32_t)h.cols};
        // tiles of consecutive rows holding about edges_per_tile edges
        rp.resize((size_t)a.rows + 1);
        if (a.rows > 0 &&
            (cudaMemcpyAsync(rp.data(), a.rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            return check_launch("gnn plan rowptr copy");
        if (a.rows > 0 && (int64_t)rp[a.rows] != a.nnz)
            return fail(GBSP_ERR_INVALID_CSR, "gnn plan: graph %d: rowptr[n] != nnz", g);
        int32_t r0 = 0;
        while (r0 < a.rows) {
            int32_t r1 = r0 + 1;
            while (r1 < a.rows && rp[r1 + 1] - rp[r0] <= edges_per_tile && r1 - r0 < 63) ++r1;
            tiles.push_back(Tile{g, r0, r1});
            r0 = r1;
        }
        nnz += a.nnz;
        rows += a.rows;
    }
    gbsp_gnn_plan *p = new gbsp_gnn_plan();
    cudaGetDevice(&p->device);
    p->G = G;
    p->ntiles = (int)tiles.size();
    p->nnz = nnz;
    p->rows = rows;
    int st = GBSP_OK;
    cudaStream_t cap = nullptr;
    if (cudaMalloc(&p->d_graphs, sizeof(GraphDesc) * (size_t)(G > 0 ? G : 1)) != cudaSuccess ||
        cudaMalloc(&p->d_tiles, sizeof(Tile) * (tiles.empty() ? 1 : tiles.size())) != cudaSuccess ||
        cudaMalloc(&p->d_ticket, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        gnn_free(p);
        return fail(GBSP_ERR_OOM, "gnn plan: allocation failed");
    }
    // stream-ordered uploads, complete before the host vectors go out of scope and before
    // the graph that reads them is recorded or replayed
    if ((G > 0 && cudaMemcpyAsync(p->d_graphs, graphs.data(), sizeof(GraphDesc) * G, cudaMemcpyHostToDevice, s) !=
                      cudaSuccess) ||
        (!tiles.empty() && cudaMemcpyAsync(p->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(),
                                           cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        st = check_launch("gnn plan upload");
        gnn_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "gnn plan upload");
    }
    // record: ticket reset + one persistent launch
    int per_sm = 0;
    if (softmax)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gnn_kernel<true>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gnn_kernel<false>, 256, 0);
    const int nblocks = sm_count() * (per_sm < 1 ? 1 : per_sm);
    GnnArgs args{p->d_graphs, p->d_tiles, p->ntiles, p->d_ticket};
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        st = check_launch("gnn plan stream");
        gnn_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "gnn plan stream");
    }
    bool okc = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (okc) {
        cudaMemsetAsync(p->d_ticket, 0, sizeof(unsigned), cap);
        if (p->ntiles > 0) {
            if (softmax)
                gnn_kernel<true><<<nblocks, 256, 0, cap>>>(args);
            else
                gnn_kernel<false><<<nblocks, 256, 0, cap>>>(args);
        }
        okc = cudaStreamEndCapture(cap, &p->graph) == cudaSuccess;
    }
    okc = okc && cudaGraphInstantiate(&p->exec, p->graph, 0) == cudaSuccess;
    cudaStreamDestroy(cap);
    if (!okc) {
        st = check_launch("gnn plan capture");
        gnn_free(p);
        return st ? st : fail(GBSP_ERR_CUDA, "gnn plan: graph capture failed");
    }
    *out = p;
    return ok();
}

GBSP_EXPORT int gbsp_gnn_plan_execute(const gbsp_gnn_plan *p, void *stream) {
    if (!p) return fail(GBSP_ERR_INVALID_ARG, "gnn execute: null plan");
    if (cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return check_launch("gnn execute");
    if (p->ntiles > 0) count_launches(1);
    return ok();
}

GBSP_EXPORT int gbsp_gnn_plan_info(const gbsp_gnn_plan *p, int64_t *info, int n) {
    if (!p || !info || n < 4) return fail(GBSP_ERR_INVALID_ARG, "gnn info: need room for 4 values");
    info[0] = p->G;
    info[1] = p->ntiles;
    info[2] = p->rows;
    info[3] = p->nnz;
    return ok();
}

GBSP_EXPORT void gbsp_gnn_plan_destroy(gbsp_gnn_plan *p) { gnn_free(p); }

GBSP_EXPORT int gbsp_gnn_plan_create(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E,
                                     gbsp_dense *O, int32_t edges_per_tile, void *stream, gbsp_gnn_plan **out) {
    return gbsp_gnn_plan_create_ex(G, S, H, E, O, edges_per_tile, 0, stream, out);
}

namespace {

int gnn_one_shot(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O, int32_t flags,
                 void *stream) {
    gbsp_gnn_plan *p = nullptr;
    int st = gbsp_gnn_plan_create_ex(G, S, H, E, O, 0, flags, stream, &p);
    if (st) return st;
    st = gbsp_gnn_plan_execute(p, stream);
    if (!st && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        st = check_launch("gnn batched");
    gnn_free(p);
    return st ? st : ok();
}

}  // namespace

GBSP_EXPORT int gnn_sddmm_spmm_batched(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E,
                                       gbsp_dense *O, void *stream) {
    return gnn_one_shot(G, S, H, E, O, 0, stream);
}

GBSP_EXPORT int gnn_gat_batched(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O,
                                void *stream) {
    return gnn_one_shot(G, S, H, E, O, GBSP_GNN_SOFTMAX, stream);
}

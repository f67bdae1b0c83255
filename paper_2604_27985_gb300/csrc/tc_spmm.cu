// Condensed-tile tensor-core SpMM: the dense 16 x 8 blocks of A run on tcgen05, the rest of
// A on the CSR kernels.
//
// Plan (once per sparsity pattern): A is cut into windows of 16 rows and each window into
// aligned 16 x 8 blocks; a block holding at least `threshold` stored entries is dense.  A
// window's dense blocks, in column order and padded to a whole pipeline stage (8 BF16 or
// 16 E4M3 blocks), form a condensed 16 x Kc tile of A (Kc = 8 * blocks) stored in the
// shared-memory image that the MMA reads (K-major, 128-byte swizzle, 16 rows x 128 bytes
// per stage).  The remaining entries form a residual CSR matrix.
//
// Execute: the residual SpMM writes C; then one CTA per window with dense blocks computes
//   C_w^T (N x 16) = B_g^T (N x Kc) * A_w^T (Kc x 16)
// with tcgen05.mma (kind::f16 for BF16, kind::f8f6f4 for E4M3; FP32 accumulation in TMEM):
// the feature dimension is the MMA's M (128 per tile, up to 4 tiles), the 16 window rows
// its N, the condensed columns its K.  B_g, the B rows of the dense blocks, is gathered by
// TMA (one copy per block) straight into the MMA's MN-major layout (8 rows x 128 bytes per
// 1 KB swizzled atom; rows past K are zero-filled, which also serves the padding blocks);
// the value tile of each stage arrives by one bulk copy.  The epilogue reads TMEM and adds
// the window's 16 rows into C.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace gbsp {

int device_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);

namespace tc {

constexpr int kBR = 16;        // rows of a dense block (= rows of a window)
constexpr int kBC = 8;         // columns of a dense block
constexpr int kATile = 2048;   // bytes of one stage of window values: 16 rows x 128 bytes
// Dense blocks per pipeline stage: 8 for BF16 (64 condensed columns), 16 for E4M3 (128).
template <bool FP8>
constexpr int blocks_per_stage() { return FP8 ? 16 : 8; }
constexpr uint64_t kWaitNs = 1000000000ull;  // a bounded wait gives up after one second

// ---- PTX wrappers ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// One box of a 3-D view of B: (128-byte feature atoms, rows, atoms) with the atoms
// outermost, so one copy lands a dense block's 8 rows as NFA consecutive 1 KB MN-major atoms.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 TMEM lanes (one per thread of the warp) x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (128-byte swizzle): start address, leading and stride
// byte offsets (all >> 4), descriptor version 1, swizzle mode 2 in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptors: FP32 accumulator, A MN-major (feature-contiguous B rows), B
// K-major (condensed window rows), M = 128, N = 16; kind::f16 with BF16 A and B (format 1),
// kind::f8f6f4 with E4M3 A and B (format 0).
constexpr uint32_t kIdescBf16 =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescE4m3 = (1u << 4) | (1u << 15) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

struct TcArgs {
    const int32_t *win_row0;  // first row of each window that has dense blocks
    const int32_t *win_blk;   // [nwin + 1] offsets of each window's (padded) dense blocks
    const int32_t *blk_col;   // block-column index of each dense block, -1 for padding
    const uint8_t *atiles;    // 2 KB swizzled value tiles, one per 8 dense blocks
    float *C;
    int64_t ldc;
    int M, K, N;
    int *err;       // set on a timed-out wait
    int block_box;  // 1: the tensor map is the 3-D atom view (one copy per block); 0: 2-D
    int withhold;   // testing the timeout path: window 0 never loads this chunk (-1: off)
    const float *wscale;  // E4M3: scale of each window row's requantised values, else null
};

template <int NT, bool FP8>
struct TcShape {
    static constexpr int BPS = blocks_per_stage<FP8>();     // dense blocks per stage
    static constexpr int NFA = FP8 ? NT : 2 * NT;           // 128-byte feature atoms per 8-row group
    static constexpr int BT = BPS * NFA * 1024;             // gathered B bytes per stage
    static constexpr int STAGE = BT + kATile;               // bytes per stage
    static constexpr int S = 2;  // stages per CTA: the next stage is copied while this one multiplies
    static constexpr int NCOLS = NT <= 2 ? 32 : 64;         // TMEM columns (16 per feature tile)
    static constexpr int SMEM = S * STAGE + 1024 + 256;     // + alignment slack + barriers
};

constexpr int kTcThreads = 128;  // 4 warps: warp 0 loads, warp 1 lane 0 issues MMAs, all 4 read TMEM
constexpr int kIssuers = 16;     // lanes of warp 0 that issue the TMA copies

template <int NT, bool FP8>
__global__ void __launch_bounds__(kTcThreads) tc_window_kernel(const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
    using SH = TcShape<NT, FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SH::S * SH::STAGE);
    uint64_t *empty = full + SH::S;
    uint64_t *done = empty + SH::S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    const int b0 = a.win_blk[w], b1 = a.win_blk[w + 1];
    const int nch = (b1 - b0) / SH::BPS;
    const int row0 = a.win_row0[w];

    if (tid == 0) {
        for (int s = 0; s < SH::S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    if (warp == 0) tmem_alloc(tslot, SH::NCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = *tslot;

    // Warp 0 produces (TMA), warp 1 issues the MMAs; each runs ahead as far as the stages
    // allow.  Four lanes of warp 0 issue a stage's block copies between them (lane 0 first
    // arms the stage's barrier and copies the value tile); their barrier waits are decided
    // together so the four stay in step.  (Gathering the rows with 16-byte copies from four
    // producer warps instead measured 1.9x slower than one TMA copy per block.)
    if (warp == 0 && lane < kIssuers) {
        static_assert(SH::BPS <= kIssuers, "one block per issuing lane and stage");
        constexpr unsigned kMask = (1u << kIssuers) - 1u;
        bool ok = true;
        int issued = 0;
        // lane kb copies block kb of every stage: its column for the first stage now, each
        // next one loaded while the current stage is in flight (no dependent load before a copy)
        int col = lane < SH::BPS && lane < b1 - b0 ? a.blk_col[b0 + lane] : -1;
        for (int ch = 0; ch < nch; ++ch) {
            const int s = ch % SH::S;
            if (ch >= SH::S) {  // stage's MMAs done
                const bool got = mbar_wait(&empty[s], ((ch / SH::S) - 1) & 1);
                if (!__all_sync(kMask, got)) {
                    ok = false;
                    break;
                }
            }
            uint8_t *bt = smem + s * SH::STAGE;
            const int qn = (ch + 1) * SH::BPS + lane;
            const int col_next = lane < SH::BPS && qn < b1 - b0 ? a.blk_col[b0 + qn] : -1;
            if (ch == a.withhold && blockIdx.x == 0) {  // nothing will complete full[s]
                col = col_next;
                continue;
            }
            if (lane == 0) {
                mbar_expect_tx(&full[s], SH::STAGE);
                bulk_load(bt + SH::BT, a.atiles + (size_t)(b0 / SH::BPS + ch) * kATile, kATile, &full[s]);
            }
            __syncwarp(kMask);
            if (lane < SH::BPS) {
                const int kb = lane;
                const int y = col >= 0 ? col * kBC : a.K;  // padding block: rows past K read as zeros
                if (a.block_box) {
                    tma_load_3d(bt + kb * SH::NFA * 1024, &tmB, &full[s], 0, y, (int)blockIdx.y * SH::NFA);
                } else {
#pragma unroll
                    for (int fa = 0; fa < SH::NFA; ++fa)
                        tma_load_2d(bt + (kb * SH::NFA + fa) * 1024, &tmB, &full[s],
                                    (FP8 ? 128 : 64) * ((int)blockIdx.y * SH::NFA + fa), y);
                }
            }
            col = col_next;
            issued = ch + 1;
        }
        if (!ok && lane == 0) atomicExch(a.err, 1);
        // every issued copy lands before the CTA can leave (bounded waits)
        if (lane == 0)
            for (int ch = issued - SH::S > 0 ? issued - SH::S : 0; ch < issued; ++ch)
                mbar_wait(&full[ch % SH::S], (ch / SH::S) & 1);
    } else if (tid == 32) {
        bool ok = true;
        for (int i = 0; i < nch; ++i) {
            const int s = i % SH::S;
            if (!mbar_wait(&full[s], (i / SH::S) & 1)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const uint32_t bt = smem_u32(smem + s * SH::STAGE);
            const uint32_t at = bt + SH::BT;
            // 4 K-steps per stage: 16 BF16 or 32 E4M3 condensed columns (32 bytes of the value
            // rows, 2 or 4 eight-row atoms of the gathered B rows) each
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t bdesc = smem_desc(at + j * 32, 16, 1024);
#pragma unroll
                for (int h = 0; h < NT; ++h) {
                    const int atom = FP8 ? (4 * j) * SH::NFA + h : (2 * j) * SH::NFA + 2 * h;
                    const uint64_t adesc = smem_desc(bt + atom * 1024, 1024, SH::NFA * 1024);
                    if constexpr (FP8)
                        mma_e4m3(taddr + h * 16, adesc, bdesc, kIdescE4m3, (i > 0 || j > 0) ? 1u : 0u);
                    else
                        mma_bf16(taddr + h * 16, adesc, bdesc, kIdescBf16, (i > 0 || j > 0) ? 1u : 0u);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
        if (!ok) atomicExch(a.err, 1);
    }
    __syncwarp();
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (features), 16 columns per tile
    const bool have = mbar_wait(done, 0);
    fence_after_sync();
    if (!have) {
        if (lane == 0) atomicExch(a.err, 2);
    } else {
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * 16), v);
            const int f = 128 * ((int)blockIdx.y * NT + h) + 32 * warp + lane;
            if (f < a.N) {
#pragma unroll
                for (int r = 0; r < kBR; ++r) {
                    const int row = row0 + r;
                    const float sc = FP8 ? __ldg(a.wscale + (int64_t)w * kBR + r) : 1.0f;
                    if (row < a.M) a.C[(int64_t)row * a.ldc + f] += v[r] * sc;
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, SH::NCOLS);
}

// ---- plan kernels ---------------------------------------------------------------------------

// cnt[w * nbc + bc] += 1 for each stored entry of window w in block column bc; also flags
// rows whose column indices are not strictly increasing.
__global__ void count_blocks_kernel(const int32_t *rowptr, const int32_t *colidx, int M, int nbc, int32_t *cnt,
                                    int *unsorted) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    int32_t *c = cnt + (int64_t)(row / kBR) * nbc;
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        const int col = colidx[p];
        atomicAdd(c + col / kBC, 1);
        if (p > p0 && colidx[p - 1] >= col) atomicExch(unsorted, 1);
    }
}

// Per window: block columns with at least `threshold` entries become dense blocks, numbered
// in column order (cnt is overwritten with the slot number, or -1).
__global__ void __launch_bounds__(256) mark_dense_kernel(int32_t *cnt, int nbc, int threshold, int32_t *win_nb) {
    __shared__ int32_t warp_tot[8];
    __shared__ int32_t carry;
    const int w = blockIdx.x;
    int32_t *c = cnt + (int64_t)w * nbc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < nbc; b += 256) {
        const int bc = b + threadIdx.x;
        const int dense = (bc < nbc && c[bc] >= threshold) ? 1 : 0;
        const unsigned bal = __ballot_sync(FULL, dense);
        const int before_in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = carry;
        for (int q = 0; q < warp; ++q) before += warp_tot[q];
        if (bc < nbc) c[bc] = dense ? before + before_in_warp : -1;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int q = 0; q < 8; ++q) t += warp_tot[q];
            carry += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) win_nb[w] = carry;
}

__global__ void pad_counts_kernel(const int32_t *win_nb, int nwin, int bps, int32_t *padded, int32_t *has) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwin) return;
    const int n = win_nb[w];
    padded[w] = (n + bps - 1) / bps * bps;
    has[w] = n > 0 ? 1 : 0;
}

// Block columns of each window's dense blocks, padding slots, and the compact window list.
__global__ void __launch_bounds__(256) fill_blocks_kernel(const int32_t *slot, int nbc, const int32_t *win_off,
                                                          const int32_t *win_nb, const int32_t *tc_index,
                                                          int32_t *blk_col, int32_t *tc_row0, int32_t *tc_blk) {
    const int w = blockIdx.x;
    const int nb = win_nb[w];
    if (nb == 0) return;
    const int off = win_off[w];
    const int npad = win_off[w + 1] - off;
    const int32_t *s = slot + (int64_t)w * nbc;
    for (int bc = threadIdx.x; bc < nbc; bc += blockDim.x)
        if (s[bc] >= 0) blk_col[off + s[bc]] = bc;
    for (int q = nb + threadIdx.x; q < npad; q += blockDim.x) blk_col[off + q] = -1;
    if (threadIdx.x == 0) {
        const int t = tc_index[w];
        tc_row0[t] = w * kBR;
        tc_blk[t] = off;
        tc_blk[t + 1] = off + npad;  // the next window writes the same value as its start
    }
}

// Byte offset of byte b of row r of a 16 x 128-byte value tile in the K-major
// 128-byte-swizzled image: 8-row atoms of 1 KB, 128 B per row, 16-byte chunks XOR-ed with
// the row in the atom.  (BF16: b = 2k for condensed column k; E4M3: b = k.)
__device__ __forceinline__ int atile_offset(int r, int b) {
    return (r >> 3) * 1024 + (r & 7) * 128 + (((b >> 4) ^ (r & 7)) << 4) + (b & 15);
}

// Scatters the entries of dense blocks into the swizzled value tiles (BF16 values, or the
// E4M3 codes that each execution folds with B's row scales and requantises) and counts the
// rest per row.  For the SDDMM it also records, per dense block and block row, the CSR
// position of the row's first entry in the block (bstart) and which of the 8 columns are
// stored (bmask; a row's entries in one block are consecutive in CSR order).
template <bool FP8>
__global__ void fill_values_kernel(const int32_t *rowptr, const int32_t *colidx, const void *vals, int M, int nbc,
                                   const int32_t *slot, const int32_t *win_off, uint8_t *tiles, int32_t *res_len,
                                   int32_t *bstart, uint32_t *bmask) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    const int w = row / kBR, r = row % kBR;
    const int32_t *s = slot + (int64_t)w * nbc;
    const int off = win_off[w];
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    int resid = 0;
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        const int col = colidx[p];
        const int sl = s[col / kBC];
        if (sl >= 0) {
            const int blk = off + sl;
            atomicOr(bmask + (int64_t)blk * kBR + r, 1u << (col % kBC));
            if (p == p0 || colidx[p - 1] / kBC != col / kBC) bstart[(int64_t)blk * kBR + r] = (int32_t)p;
            if constexpr (FP8) {
                const int k = (blk % 16) * kBC + col % kBC;
                tiles[(int64_t)(blk / 16) * kATile + atile_offset(r, k)] = static_cast<const uint8_t *>(vals)[p];
            } else {
                const int k = (blk % 8) * kBC + col % kBC;
                uint8_t *tile = tiles + (int64_t)(blk / 8) * kATile;
                *reinterpret_cast<uint16_t *>(tile + atile_offset(r, 2 * k)) = static_cast<const uint16_t *>(vals)[p];
            }
        } else {
            ++resid;
        }
    }
    for (int o = 16; o > 0; o >>= 1) resid += __shfl_xor_sync(FULL, resid, o);
    if (lane == 0) res_len[row] = resid;
}

// Copies the residual entries of each row, in order, to the residual CSR, with each one's
// position in A's CSR (for the SDDMM, whose values and outputs are in that order).
template <typename T>
__global__ void fill_residual_kernel(const int32_t *rowptr, const int32_t *colidx, const T *vals, int M, int nbc,
                                     const int32_t *slot, const int32_t *res_ptr, int32_t *res_col, T *res_val,
                                     int32_t *res_pos) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    const int32_t *s = slot + (int64_t)(row / kBR) * nbc;
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    int64_t out = res_ptr[row];
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t p = base + lane;
        int col = 0;
        bool keep = false;
        if (p < p1) {
            col = colidx[p];
            keep = s[col / kBC] < 0;
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) {
            const int64_t q = out + __popc(bal & ((1u << lane) - 1u));
            res_col[q] = col;
            res_val[q] = vals[p];
            res_pos[q] = (int32_t)p;
        }
        out += __popc(bal);
    }
}

// E4M3 execution, before the window kernel: for each window row r, a~_k = (s_i q_ik) t_col(k)
// in FP32 over its condensed columns (B's per-row scale folded into A, since a scale along
// the contraction cannot be applied after the MMA); u_r = 2^e with e the smallest exponent
// (at least -126) for which max |a~| <= 448 u_r (1 for an empty row); the E4M3 rounding
// (nearest-even, saturating) of a~ / u_r goes into the swizzled tiles and u_r to the
// epilogue.  A power of two makes the division exact, so a~ already on the E4M3 grid
// (unit scales, small integers) passes through unchanged.
//
// One CTA per window.  Thread t owns bytes 8t..8t+7 of every 2 KB tile of the window: one
// row r and 8 consecutive condensed columns of one block (the swizzle permutes 16-byte
// chunks only), read from the code tiles and written to the same offsets of the output
// tiles.  The 16 threads sharing a row reduce its maximum with shuffles; the values are
// recomputed in the second pass rather than held.
__device__ __forceinline__ void fold_load_t(const float *b_scale, int col, int K, bool vec_ok, float (&t)[8]) {
    const int64_t k0 = (int64_t)col * kBC;
    if (col >= 0 && vec_ok && k0 + 8 <= K) {
        const float4 lo = __ldg(reinterpret_cast<const float4 *>(b_scale + k0));
        const float4 hi = __ldg(reinterpret_cast<const float4 *>(b_scale + k0) + 1);
        t[0] = lo.x, t[1] = lo.y, t[2] = lo.z, t[3] = lo.w, t[4] = hi.x, t[5] = hi.y, t[6] = hi.z, t[7] = hi.w;
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) t[c] = (col >= 0 && k0 + c < K) ? __ldg(b_scale + k0 + c) : 0.f;
    }
}

__global__ void __launch_bounds__(256) fold_e4m3_kernel(const uint8_t *__restrict__ qtiles,
                                                        const float *__restrict__ a_scale,
                                                        const int32_t *__restrict__ tc_row0,
                                                        const int32_t *__restrict__ tc_blk,
                                                        const int32_t *__restrict__ blk_col,
                                                        const float *__restrict__ b_scale, int M, int K, int vec_ok,
                                                        uint8_t *__restrict__ atiles, float *__restrict__ wscale) {
    const int w = blockIdx.x, t = threadIdx.x;
    const int b0 = tc_blk[w], ntiles = (tc_blk[w + 1] - b0) / 16;
    const int rowin = (t >> 4) & 7, r = (t >> 7) * 8 + rowin;
    const int kb = ((((t & 15) >> 1) ^ rowin) * 16 + 8 * (t & 1)) >> 3;  // block of the tile
    const int row = tc_row0[w] + r;
    const float s = row < M ? __ldg(a_scale + row) : 0.f;
    // two codes decoded per conversion and two products per packed FP32 multiply (the same
    // single roundings as scalar code)
    auto values = [&](int tile, float (&v)[8]) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(qtiles + (int64_t)(b0 / 16 + tile) * kATile) + t);
        float tk[8];
        fold_load_t(b_scale, __ldg(blk_col + b0 + tile * 16 + kb), K, vec_ok != 0, tk);
        const float2 s2 = make_float2(s, s);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t word = h < 2 ? q.x : q.y;
            const float2 d = E4M3::pair((uint16_t)(word >> (16 * (h & 1))));
            const float2 r = __fmul2_rn(__fmul2_rn(s2, d), make_float2(tk[2 * h], tk[2 * h + 1]));
            v[2 * h] = r.x;
            v[2 * h + 1] = r.y;
        }
    };
    float amax = 0.f;
#pragma unroll 4
    for (int tile = 0; tile < ntiles; ++tile) {
        float v[8];
        values(tile, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) amax = fmaxf(amax, fabsf(v[c]));
    }
    for (int off = 8; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    int e = 0;
    if (amax > 0.f) {
        int E;
        const float m = frexpf(amax, &E);  // amax = m 2^E, m in [0.5, 1); 448 = 0.875 2^9
        e = max(m <= 0.875f ? E - 9 : E - 8, -126);
    }
    if ((t & 15) == 0) wscale[(int64_t)w * kBR + r] = ldexpf(1.0f, e);
    const float inv = ldexpf(1.0f, -e);
#pragma unroll 4
    for (int tile = 0; tile < ntiles; ++tile) {
        float v[8];
        values(tile, v);
        uint32_t out[2] = {0u, 0u};
        const float2 inv2 = make_float2(inv, inv);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 x = __fmul2_rn(make_float2(v[2 * h], v[2 * h + 1]), inv2);
            const uint32_t two = __nv_cvt_float2_to_fp8x2(x, __NV_SATFINITE, __NV_E4M3);  // x.x in the low byte
            out[h >> 1] |= (two & 0xffffu) << (16 * (h & 1));
        }
        reinterpret_cast<uint2 *>(atiles + (int64_t)(b0 / 16 + tile) * kATile)[t] = make_uint2(out[0], out[1]);
    }
}

// ---- condensed-tile SDDMM ------------------------------------------------------------------
//
// For a window with dense blocks, the 16 x 8 outputs of each block are one small product:
//   D (128 x 16) = Y_g (128 x Kd) X_w^T (Kd x 16)
// with Y_g the Y rows of 16 blocks' columns (8 each) and X_w the window's 16 X rows, both
// K-major (Kd contiguous) in 128-byte-swizzled shared memory; the epilogue writes
// out[p] = s_p D[j][i] only for the stored entries (Eq. 2), found from the plan's per block
// row first position and column mask.  One stage of 16 blocks at a time, its Y rows
// arriving in units of KH 128-byte K-blocks through two shared-memory slots (a slot is
// refilled once its unit's MMAs are done); two TMEM buffers let stage ch's epilogue overlap
// stage ch + 1's copies and MMAs.

constexpr int kSdBlocks = 16;  // dense blocks per stage: MMA M = 128 gathered Y rows

struct TcSddmmArgs {
    const int32_t *win_row0, *win_blk, *blk_col;
    const int32_t *bstart;
    const uint32_t *bmask;
    const float *svals;
    float *out;
    const float *x_scale, *y_scale;  // E4M3 per-row scales of X and Y, else null
    int M, Ny, KB;                   // rows of X and of Y; 128-byte K-blocks per row
    int KH;                          // K-blocks per copy unit (KB a multiple of KH)
    int *err;
};

template <bool FP8>
__global__ void __launch_bounds__(128) tc_sddmm_kernel(const __grid_constant__ CUtensorMap tmY,
                                                       const __grid_constant__ CUtensorMap tmX,
                                                       const TcSddmmArgs a) {
    constexpr uint32_t kIdesc = (1u << 4) | ((FP8 ? 0u : 1u) << 7) | ((FP8 ? 0u : 1u) << 10) | ((16u >> 3) << 17) |
                                ((128u >> 4) << 24);  // FP32 D, both operands K-major, M = 128, N = 16
    const int KH = a.KH;  // K-blocks per unit: one copy box per block covers KH 128-byte K-blocks
    const uint32_t kUnitBytes = (uint32_t)(kSdBlocks * KH * 1024);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int KB = a.KB;
    uint8_t *slots = smem;                  // [2][16 blocks][KH][8 rows][128 B]
    uint8_t *xt = smem + 2 * kUnitBytes;    // [KB][16 rows][128 B]
    uint64_t *full = reinterpret_cast<uint64_t *>(xt + 2 * KB * 1024);  // [2] per slot
    uint64_t *freed = full + 2;             // [2] per slot: its unit's MMAs are done
    uint64_t *mdone = full + 4;             // [2] per TMEM buffer: a stage's MMAs are done
    uint64_t *epi_done = full + 6;          // [2] per TMEM buffer: its epilogue has read it
    uint64_t *xfull = full + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 9);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.x;
    const int b0 = a.win_blk[w], b1 = a.win_blk[w + 1];
    const int nst = (b1 - b0 + kSdBlocks - 1) / kSdBlocks;
    const int NU = KB / KH;       // units per stage
    const int nunits = nst * NU;  // unit u: stage u / NU, K-blocks (u % NU) * KH ...
    const int row0 = a.win_row0[w];
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&freed[i], 1);
            mbar_init(&mdone[i], 1);
            mbar_init(&epi_done[i], kTcThreads);
        }
        mbar_init(xfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, 32);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = *tslot;

    float xs[kBR];  // E4M3: the window rows' X scales
#pragma unroll
    for (int r = 0; r < kBR; ++r) xs[r] = FP8 && row0 + r < a.M ? __ldg(a.x_scale + row0 + r) : 1.0f;
    constexpr unsigned kMask = (1u << kIssuers) - 1u;
    // unit u's copies into slot u % 2: one TMA box per block (8 Y rows, one K-block); blocks
    // past the window's end and padding blocks read rows past Y's end, which arrive as zeros
    auto issue_unit = [&](int u) {
        const int ch = u / NU, kb = (u % NU) * KH;
        if (lane == 0) mbar_expect_tx(&full[u & 1], kUnitBytes);
        __syncwarp(kMask);
        for (int q = lane; q < kSdBlocks; q += kIssuers) {
            const int blk = b0 + ch * kSdBlocks + q;
            const int col = blk < b1 ? a.blk_col[blk] : -1;
            tma_load_3d(slots + (u & 1) * kUnitBytes + q * KH * 1024, &tmY, &full[u & 1], 0,
                        col >= 0 ? col * kBC : a.Ny, kb);
        }
    };
    const bool producer = warp == 0 && lane < kIssuers;
    if (producer) {
        if (lane == 0) {
            mbar_expect_tx(xfull, (uint32_t)(2 * KB * 1024));
            tma_load_3d(xt, &tmX, xfull, 0, row0, 0);
        }
        for (int u = 0; u < 2 && u < nunits; ++u) issue_unit(u);
    }
    bool ok = true;
    bool x_landed = false;
    int unlanded = -1;  // a unit whose copies the MMA thread gave up waiting for
    for (int ch = 0; ch < nst; ++ch) {
        const int buf = ch & 1;
        for (int h = 0; h < NU; ++h) {
            const int u = ch * NU + h;
            if (tid == 32) {
                if (!x_landed) x_landed = mbar_wait(xfull, 0);
                const bool landed = mbar_wait(&full[u & 1], (u >> 1) & 1);
                if (!landed) unlanded = u;
                bool go = x_landed && landed && ok;
                if (go && h == 0 && ch >= 2) go = mbar_wait(&epi_done[buf], ((ch >> 1) - 1) & 1);
                if (!go) {
                    if (ok) atomicExch(a.err, 3);
                    ok = false;
                } else {
                    fence_after_sync();
                    const uint32_t sa = smem_u32(slots + (u & 1) * kUnitBytes), sx = smem_u32(xt);
                    for (int kk = 0; kk < KH; ++kk) {
                        const int kb = h * KH + kk;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint64_t adesc = smem_desc(sa + kk * 1024 + j * 32, 16, KH * 1024);
                            const uint64_t bdesc = smem_desc(sx + kb * 2048 + j * 32, 16, 1024);
                            const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
                            if constexpr (FP8)
                                mma_e4m3(taddr + buf * 16, adesc, bdesc, kIdesc, acc);
                            else
                                mma_bf16(taddr + buf * 16, adesc, bdesc, kIdesc, acc);
                        }
                    }
                }
                mma_commit(&freed[u & 1]);  // also when skipped, so the waits end
                if (h == NU - 1) mma_commit(&mdone[buf]);
            }
            // the slot of unit u is refilled with unit u + 2 once unit u's MMAs are done
            if (producer && u + 2 < nunits) {
                const bool got = mbar_wait(&freed[u & 1], (u >> 1) & 1);
                if (__all_sync(kMask, got)) issue_unit(u + 2);
                else if (lane == 0) atomicExch(a.err, 5);
            }
        }
        __syncwarp();
        const bool have = mbar_wait(&mdone[buf], (ch >> 1) & 1);  // this stage's MMAs are done
        fence_after_sync();
        if (!have && lane == 0) atomicExch(a.err, 4);
        __syncwarp();
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * 16), v);
        const int m = 32 * warp + lane;  // gathered Y row: block m / 8, column m % 8
        const int blk = b0 + ch * kSdBlocks + (m >> 3), c = m & 7;
        const int col = have && ok && blk < b1 ? a.blk_col[blk] : -1;
        if (col >= 0) {
            // the block's 16 row masks and first positions in four 16-byte loads each, then
            // every stored entry's value, then the stores: two memory latencies per stage
            uint4 mk4[4], st4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                mk4[i] = __ldg(reinterpret_cast<const uint4 *>(a.bmask + (int64_t)blk * kBR) + i);
                st4[i] = __ldg(reinterpret_cast<const uint4 *>(a.bstart + (int64_t)blk * kBR) + i);
            }
            const int64_t j = (int64_t)col * kBC + c;  // past Y's end in a ragged last block column
            const float ys = FP8 && j < a.Ny ? __ldg(a.y_scale + j) : 1.0f;
            int64_t pos[kBR];
            float sv[kBR];
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                const uint4 &mq = mk4[r >> 2], &sq = st4[r >> 2];
                const uint32_t mk = (r & 3) == 0 ? mq.x : (r & 3) == 1 ? mq.y : (r & 3) == 2 ? mq.z : mq.w;
                const uint32_t st = (r & 3) == 0 ? sq.x : (r & 3) == 1 ? sq.y : (r & 3) == 2 ? sq.z : sq.w;
                pos[r] = ((mk >> c) & 1u) ? (int64_t)(int32_t)st + __popc(mk & ((1u << c) - 1u)) : -1;
                sv[r] = pos[r] >= 0 ? __ldg(a.svals + pos[r]) : 0.f;
            }
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                if (pos[r] < 0) continue;
                float val = sv[r] * v[r];
                if (FP8) val *= xs[r] * ys;
                a.out[pos[r]] = val;
            }
        }
        fence_before_sync();
        mbar_arrive(&epi_done[buf]);
    }
    // copies the MMA thread gave up on (after a timeout) land before the CTA leaves
    if (tid == 32) {
        if (unlanded >= 0) mbar_wait(&full[unlanded & 1], (unlanded >> 1) & 1);
        if (!x_landed) mbar_wait(xfull, 0);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 32);
}

}  // namespace tc
}  // namespace gbsp

// ---- plan object and entry points -----------------------------------------------------------

using namespace gbsp;
using namespace gbsp::tc;

struct gbsp_plan {
    int device;
    int dtype;           // GBSP_BF16 or GBSP_E4M3
    int64_t M, K, nnz;
    int threshold;
    int nwin_tc;         // windows with dense blocks
    int64_t nblocks;     // dense blocks, padded per window to a stage (8 BF16, 16 E4M3 blocks)
    int64_t dense_nnz;   // stored entries inside dense blocks
    int64_t res_nnz;     // residual entries
    int32_t *tc_row0, *tc_blk, *blk_col;
    uint8_t *atiles;     // swizzled value tiles (E4M3: rewritten by each execution)
    uint8_t *qtiles;     // E4M3: A's codes in the same tile layout
    float *wscale;       // E4M3: per window row scale of the requantised tiles
    float *res_scale;    // E4M3: A's row scales (the residual's)
    int32_t *bstart;     // per dense block and block row: CSR position of its first entry
    uint32_t *bmask;     // per dense block and block row: stored columns (8 bits)
    int32_t *res_pos;    // per residual entry: its CSR position in A
    int32_t *rowptr_full, *colidx_full;  // A's pattern, for an SDDMM that skips the tiles
    int32_t *res_rowptr, *res_colidx;
    void *res_vals;
    int *err;
    int withhold;  // see gbsp_plan_test_withhold
    gbsp_opts residual_opts;
    int residual_auto;  // the split AUTO chose for the residual at creation (0: not measured)
};

namespace {

template <class T>
int dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(GBSP_ERR_OOM, "plan: allocation of %zu bytes failed", count * sizeof(T));
    }
    return GBSP_OK;
}

void plan_free(gbsp_plan *p) {
    if (!p) return;
    cudaFree(p->tc_row0);
    cudaFree(p->tc_blk);
    cudaFree(p->blk_col);
    cudaFree(p->atiles);
    cudaFree(p->qtiles);
    cudaFree(p->wscale);
    cudaFree(p->res_scale);
    cudaFree(p->res_rowptr);
    cudaFree(p->res_colidx);
    cudaFree(p->res_vals);
    cudaFree(p->bstart);
    cudaFree(p->bmask);
    cudaFree(p->res_pos);
    cudaFree(p->rowptr_full);
    cudaFree(p->colidx_full);
    cudaFree(p->err);
    delete p;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <int NT, bool FP8>
int launch_tc(const CUtensorMap &map, const TcArgs &args, int nwin, int ngroups, cudaStream_t s) {
    using SH = TcShape<NT, FP8>;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(GBSP_ERR_UNSUPPORTED, "tc: device ordinal %d", dev);
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(tc_window_kernel<NT, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM) !=
            cudaSuccess)
            return check_launch("tc smem attribute");
        attr_set[dev] = true;
    }
    tc_window_kernel<NT, FP8><<<dim3((unsigned)nwin, (unsigned)ngroups), kTcThreads, SH::SMEM, s>>>(map, args);
    count_launches(1);
    return check_launch("tc window kernel");
}

}  // namespace

GBSP_EXPORT int gbsp_plan_create(const gbsp_csr *A, int32_t threshold, const gbsp_opts *residual_opts, void *stream,
                                 gbsp_plan **out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "plan: null output");
    *out = nullptr;
    if (!A || A->rows < 0 || A->cols < 0 || A->nnz < 0 || A->rows > 2147483647LL || A->cols > 2147483647LL)
        return fail(GBSP_ERR_INVALID_ARG, "plan: bad CSR descriptor");
    if (A->dtype != GBSP_BF16 && A->dtype != GBSP_E4M3)
        return fail(GBSP_ERR_UNSUPPORTED, "plan: the tensor-core path takes BF16 or E4M3 values");
    if (A->dtype == GBSP_E4M3 && A->rows > 0 && !A->row_scale)
        return fail(GBSP_ERR_INVALID_ARG, "plan: E4M3 values need row scales");
    if (A->rows > 0 && !A->rowptr) return fail(GBSP_ERR_INVALID_ARG, "plan: null rowptr");
    if (A->nnz > 0 && (!A->colidx || !A->vals)) return fail(GBSP_ERR_INVALID_ARG, "plan: null colidx / vals");
    // defaults measured on 16,384^2 at 90% (N = 256), uniform and clustered: the E4M3 residual
    // runs on ALU-bound CSR kernels, so sparser blocks still pay on the tensor cores
    if (threshold < 1) threshold = A->dtype == GBSP_E4M3 ? 10 : 14;
    const int64_t M = A->rows, K = A->cols;
    const int64_t nwin = (M + kBR - 1) / kBR, nbc = (K + kBC - 1) / kBC;
    if (nwin * nbc > (int64_t)1 << 28)
        return fail(GBSP_ERR_UNSUPPORTED, "plan: %lld windows x %lld block columns exceed the block map",
                    (long long)nwin, (long long)nbc);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp8 = A->dtype == GBSP_E4M3;
    const int bps = fp8 ? blocks_per_stage<true>() : blocks_per_stage<false>();
    gbsp_plan *p = new gbsp_plan();
    cudaGetDevice(&p->device);
    p->dtype = A->dtype;
    p->M = M;
    p->K = K;
    p->nnz = A->nnz;
    p->threshold = threshold;
    p->residual_opts = residual_opts ? *residual_opts : gbsp_opts{};
    p->withhold = -1;
    int st = GBSP_OK;
    int32_t *slot = nullptr, *win_nb = nullptr, *padded = nullptr, *has = nullptr, *win_off = nullptr,
            *tc_index = nullptr, *res_len = nullptr;
    int *flag = nullptr;
    int32_t totals[2] = {0, 0};
    int hflag = 0;
    const unsigned row_blocks = (unsigned)((M + 7) / 8);
#define GBSP_TRY(x)              \
    do {                         \
        if ((st = (x))) goto out; \
    } while (0)
    GBSP_TRY(dev_alloc(&slot, (size_t)(nwin * nbc)));
    GBSP_TRY(dev_alloc(&win_nb, (size_t)nwin + 1));
    GBSP_TRY(dev_alloc(&padded, (size_t)nwin + 1));
    GBSP_TRY(dev_alloc(&has, (size_t)nwin + 1));
    GBSP_TRY(dev_alloc(&win_off, (size_t)nwin + 1));
    GBSP_TRY(dev_alloc(&tc_index, (size_t)nwin + 1));
    GBSP_TRY(dev_alloc(&res_len, (size_t)M + 1));
    GBSP_TRY(dev_alloc(&flag, 1));
    GBSP_TRY(dev_alloc(&p->err, 1));
    cudaMemsetAsync(slot, 0, sizeof(int32_t) * (size_t)(nwin * nbc), s);
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    cudaMemsetAsync(p->err, 0, sizeof(int), s);
    if (M > 0) {
        count_blocks_kernel<<<row_blocks, 256, 0, s>>>(A->rowptr, A->colidx, (int)M, (int)nbc, slot, flag);
        mark_dense_kernel<<<(unsigned)nwin, 256, 0, s>>>(slot, (int)nbc, threshold, win_nb);
        pad_counts_kernel<<<(unsigned)((nwin + 255) / 256), 256, 0, s>>>(win_nb, (int)nwin, bps, padded, has);
        count_launches(3);
        GBSP_TRY(check_launch("plan count"));
    }
    GBSP_TRY(device_exclusive_scan(padded, win_off, nwin, s));
    GBSP_TRY(device_exclusive_scan(has, tc_index, nwin, s));
    cudaMemcpyAsync(&totals[0], win_off + nwin, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&totals[1], tc_index + nwin, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) GBSP_TRY(check_launch("plan sync"));
    if (hflag) GBSP_TRY(fail(GBSP_ERR_UNSUPPORTED, "plan: column indices must be strictly increasing in every row"));
    p->nblocks = totals[0];
    p->nwin_tc = totals[1];
    GBSP_TRY(dev_alloc(&p->blk_col, (size_t)p->nblocks));
    GBSP_TRY(dev_alloc(&p->atiles, (size_t)(p->nblocks / bps) * kATile));
    GBSP_TRY(dev_alloc(&p->tc_row0, (size_t)p->nwin_tc));
    GBSP_TRY(dev_alloc(&p->tc_blk, (size_t)p->nwin_tc + 1));
    cudaMemsetAsync(p->atiles, 0, (size_t)(p->nblocks / bps) * kATile, s);
    cudaMemsetAsync(p->tc_blk, 0, sizeof(int32_t), s);
    if (fp8) {
        GBSP_TRY(dev_alloc(&p->qtiles, (size_t)(p->nblocks / bps) * kATile));
        GBSP_TRY(dev_alloc(&p->wscale, (size_t)p->nwin_tc * kBR));
        GBSP_TRY(dev_alloc(&p->res_scale, (size_t)M));
        cudaMemsetAsync(p->qtiles, 0, (size_t)(p->nblocks / bps) * kATile, s);
        if (M > 0) cudaMemcpyAsync(p->res_scale, A->row_scale, sizeof(float) * (size_t)M, cudaMemcpyDeviceToDevice, s);
    }
    GBSP_TRY(dev_alloc(&p->bstart, (size_t)p->nblocks * kBR));
    GBSP_TRY(dev_alloc(&p->bmask, (size_t)p->nblocks * kBR));
    cudaMemsetAsync(p->bmask, 0, sizeof(uint32_t) * (size_t)p->nblocks * kBR, s);
    if (M > 0) {
        fill_blocks_kernel<<<(unsigned)nwin, 256, 0, s>>>(slot, (int)nbc, win_off, win_nb, tc_index, p->blk_col,
                                                          p->tc_row0, p->tc_blk);
        if (fp8)
            fill_values_kernel<true><<<row_blocks, 256, 0, s>>>(A->rowptr, A->colidx, A->vals, (int)M, (int)nbc, slot,
                                                                win_off, p->qtiles, res_len, p->bstart, p->bmask);
        else
            fill_values_kernel<false><<<row_blocks, 256, 0, s>>>(A->rowptr, A->colidx, A->vals, (int)M, (int)nbc, slot,
                                                                 win_off, p->atiles, res_len, p->bstart, p->bmask);
        count_launches(2);
        GBSP_TRY(check_launch("plan fill"));
    }
    GBSP_TRY(dev_alloc(&p->res_rowptr, (size_t)M + 1));
    GBSP_TRY(device_exclusive_scan(res_len, p->res_rowptr, M, s));
    cudaMemcpyAsync(&totals[0], p->res_rowptr + M, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) GBSP_TRY(check_launch("plan sync"));
    p->res_nnz = totals[0];
    p->dense_nnz = p->nnz - p->res_nnz;
    GBSP_TRY(dev_alloc(&p->res_colidx, (size_t)p->res_nnz));
    GBSP_TRY(dev_alloc(&p->res_pos, (size_t)p->res_nnz));
    GBSP_TRY(dev_alloc(&p->rowptr_full, (size_t)M + 1));
    GBSP_TRY(dev_alloc(&p->colidx_full, (size_t)p->nnz));
    if (M > 0) cudaMemcpyAsync(p->rowptr_full, A->rowptr, sizeof(int32_t) * (size_t)(M + 1), cudaMemcpyDeviceToDevice, s);
    if (p->nnz > 0)
        cudaMemcpyAsync(p->colidx_full, A->colidx, sizeof(int32_t) * (size_t)p->nnz, cudaMemcpyDeviceToDevice, s);
    if (fp8) {
        GBSP_TRY(dev_alloc(reinterpret_cast<uint8_t **>(&p->res_vals), (size_t)p->res_nnz));
    } else {
        GBSP_TRY(dev_alloc(reinterpret_cast<uint16_t **>(&p->res_vals), (size_t)p->res_nnz));
    }
    if (M > 0) {
        if (fp8)
            fill_residual_kernel<uint8_t><<<row_blocks, 256, 0, s>>>(
                A->rowptr, A->colidx, static_cast<const uint8_t *>(A->vals), (int)M, (int)nbc, slot, p->res_rowptr,
                p->res_colidx, static_cast<uint8_t *>(p->res_vals), p->res_pos);
        else
            fill_residual_kernel<uint16_t><<<row_blocks, 256, 0, s>>>(
                A->rowptr, A->colidx, static_cast<const uint16_t *>(A->vals), (int)M, (int)nbc, slot, p->res_rowptr,
                p->res_colidx, static_cast<uint16_t *>(p->res_vals), p->res_pos);
        count_launches(1);
        GBSP_TRY(check_launch("plan residual"));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) GBSP_TRY(check_launch("plan sync"));
    if (p->residual_opts.variant == GBSP_VARIANT_AUTO && M > 0) {
        // the residual's automatic split is measured here, where the stream is synchronised
        // anyway, so that executions never synchronise
        const gbsp_csr R{p->M, p->K, p->res_nnz, p->res_rowptr, p->res_colidx, p->res_vals, p->res_scale, p->dtype};
        // (the B of later executions is not known yet: the rule is applied as for B in L2)
        GBSP_TRY(auto_choice(R, kOpSpmm, 0, 0, s, &p->residual_auto, nullptr));
    }
out:
#undef GBSP_TRY
    cudaFree(slot);
    cudaFree(win_nb);
    cudaFree(padded);
    cudaFree(has);
    cudaFree(win_off);
    cudaFree(tc_index);
    cudaFree(res_len);
    cudaFree(flag);
    if (st) {
        plan_free(p);
        return st;
    }
    *out = p;
    return ok();
}

namespace {

// The tensor map of B's rows for the window kernel: the 3-D atom view (one copy per block:
// 128-byte feature atoms of 8 rows, atoms 128 B apart, rows ld apart) when N is a multiple
// of 128, else a 2-D map copied one 128-byte atom at a time (features past N read as zeros).
int encode_b_map(const gbsp_dense *B, int64_t K, bool fp8, int nt, CUtensorMap *map, int *block_box) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(GBSP_ERR_CUDA, "plan execute: cuTensorMapEncodeTiled is not available");
    const int64_t N = B->cols;
    const int es = fp8 ? 1 : 2, atom = 128 / es;  // elements per 128-byte atom
    const CUtensorMapDataType ty = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    *block_box = 0;
    if (N % 128 == 0) {
        const int natoms = (int)(N / atom);
        const int tile_atoms = fp8 ? 1 : 2;  // atoms of one 128-feature tile, gathered per CTA
        const cuuint64_t dims3[3] = {(cuuint64_t)atom, (cuuint64_t)K, (cuuint64_t)natoms};
        const cuuint64_t strides3[2] = {(cuuint64_t)B->ld * es, 128};
        const cuuint32_t box3[3] = {(cuuint32_t)atom, 8, (cuuint32_t)tile_atoms};
        const cuuint32_t estr3[3] = {1, 1, 1};
        *block_box = natoms == (fp8 ? nt : 2 * nt) &&
                     enc(map, ty, 3, B->data, dims3, strides3, box3, estr3, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (!*block_box) {
        const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)K};
        const cuuint64_t strides[1] = {(cuuint64_t)B->ld * es};
        const cuuint32_t box[2] = {(cuuint32_t)atom, 8};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(map, ty, 2, B->data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fail(GBSP_ERR_CUDA, "plan execute: tensor map encoding failed");
    }
    return GBSP_OK;
}

// One CTA per dense window and 128-feature tile: a window's tiles read the same value
// tiles but gather disjoint atoms of each B row and write disjoint columns of C, so
// splitting them doubles (N = 256) or quadruples (N = 512) the work items without any
// combining step; with one item per window the 1,024 windows of a 16,384-row matrix fill
// 1.35 waves of 5 CTAs per SM and leave most of the second wave's slots idle.
template <bool FP8>
int launch_tc_nt(int nt, const CUtensorMap &map, const TcArgs &args, int nwin, cudaStream_t s) {
    return launch_tc<1, FP8>(map, args, nwin, nt, s);
}

}  // namespace

GBSP_EXPORT int gbsp_plan_execute(const gbsp_plan *p, const gbsp_dense *B, gbsp_dense *C, void *stream) {
    if (!p || !B || !C) return fail(GBSP_ERR_INVALID_ARG, "plan execute: null argument");
    const bool fp8 = p->dtype == GBSP_E4M3;
    if (B->dtype != p->dtype || C->dtype != GBSP_F32)
        return fail(GBSP_ERR_UNSUPPORTED, "plan execute: B must have the plan's dtype (%s) and C be FP32",
                    fp8 ? "E4M3" : "BF16");
    if (B->rows != p->K || C->rows != p->M || C->cols != B->cols || B->ld < B->cols || C->ld < C->cols)
        return fail(GBSP_ERR_INVALID_ARG, "plan execute: shape mismatch");
    if (fp8 && B->rows > 0 && !B->row_scale) return fail(GBSP_ERR_INVALID_ARG, "plan execute: E4M3 B needs row scales");
    const int64_t N = B->cols;
    const int amul = fp8 ? 16 : 8;  // elements per 16 bytes
    if (p->nwin_tc > 0 && (N % amul || B->ld % amul || !aligned16(B->data) || N < 64 || N > 512))
        return fail(GBSP_ERR_UNSUPPORTED, "plan execute: tensor-core tiles need 64 <= N <= 512, N and ld multiples "
                                          "of %d and a 16-byte aligned B",
                    amul);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // residual entries (and the overwrite of C) through the CSR kernels
    gbsp_csr R{p->M, p->K, p->res_nnz, p->res_rowptr, p->res_colidx, p->res_vals, p->res_scale, p->dtype};
    gbsp_opts ro = p->residual_opts;
    const bool vec = aligned16(B->data) && B->ld % amul == 0 && N % amul == 0 && aligned16(C->data) && C->ld % 4 == 0;
    if (ro.variant == GBSP_VARIANT_AUTO && p->residual_auto > 0 && vec) ro.variant = p->residual_auto;
    int st = spmm_csr_ex(&R, B, C, &ro, stream);
    if (st) return st;
    if (p->nwin_tc == 0 || N == 0) return ok();
    const int nt = (int)((N + 127) / 128);
    CUtensorMap map;
    int block_box = 0;
    if ((st = encode_b_map(B, p->K, fp8, nt, &map, &block_box))) return st;
    if (fp8) {
        const float *t = static_cast<const float *>(B->row_scale);
        fold_e4m3_kernel<<<(unsigned)p->nwin_tc, 256, 0, s>>>(p->qtiles, p->res_scale, p->tc_row0, p->tc_blk,
                                                              p->blk_col, t, (int)p->M, (int)p->K, aligned16(t) ? 1 : 0,
                                                              p->atiles, p->wscale);
        count_launches(1);
        if ((st = check_launch("tc fold"))) return st;
    }
    TcArgs args{p->tc_row0, p->tc_blk, p->blk_col, p->atiles, static_cast<float *>(C->data), C->ld, (int)p->M,
                (int)p->K, (int)N, p->err, block_box, p->withhold, p->wscale};
    st = fp8 ? launch_tc_nt<true>(nt, map, args, p->nwin_tc, s) : launch_tc_nt<false>(nt, map, args, p->nwin_tc, s);
    return st ? st : ok();
}

namespace {

// 3-D atom view of a row-major matrix whose rows are `kb` whole 128-byte atoms: dims
// (atom elements, rows, atoms), a box of `box_rows` rows and `box_atoms` atoms.
int encode_atom_view(const gbsp_dense *D, bool fp8, int kb, int box_rows, int box_atoms, CUtensorMap *map) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(GBSP_ERR_CUDA, "plan sddmm: cuTensorMapEncodeTiled is not available");
    const int es = fp8 ? 1 : 2, atom = 128 / es;
    const cuuint64_t dims[3] = {(cuuint64_t)atom, (cuuint64_t)D->rows, (cuuint64_t)kb};
    const cuuint64_t strides[2] = {(cuuint64_t)D->ld * es, 128};
    const cuuint32_t box[3] = {(cuuint32_t)atom, (cuuint32_t)box_rows, (cuuint32_t)box_atoms};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, D->data, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(GBSP_ERR_CUDA, "plan sddmm: tensor map encoding failed");
    return GBSP_OK;
}

template <bool FP8>
int launch_tc_sddmm(const CUtensorMap &my, const CUtensorMap &mx, const TcSddmmArgs &args, int nwin, cudaStream_t s) {
    constexpr int kMaxSmem = 2 * 2 * 16 * 1024 + 2 * 8 * 1024 + 1024 + 128;  // KH <= 2, KB <= 8
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(GBSP_ERR_UNSUPPORTED, "tc sddmm: device ordinal %d", dev);
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(tc_sddmm_kernel<FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
            cudaSuccess)
            return check_launch("tc sddmm smem attribute");
        attr_set[dev] = true;
    }
    const int smem = 2 * args.KH * 16 * 1024 + 2 * args.KB * 1024 + 1024 + 128;  // two unit slots, X rows, barriers
    tc_sddmm_kernel<FP8><<<nwin, kTcThreads, smem, s>>>(my, mx, args);
    count_launches(1);
    return check_launch("tc sddmm kernel");
}

}  // namespace

GBSP_EXPORT int gbsp_plan_sddmm(const gbsp_plan *p, const float *svals, const gbsp_dense *X, const gbsp_dense *Y,
                                float *out, int32_t tiles, void *stream) {
    if (!p || !X || !Y) return fail(GBSP_ERR_INVALID_ARG, "plan sddmm: null argument");
    if (p->nnz > 0 && (!svals || !out)) return fail(GBSP_ERR_INVALID_ARG, "plan sddmm: null svals / out");
    if (X->dtype != Y->dtype || (X->dtype != GBSP_BF16 && X->dtype != GBSP_E4M3))
        return fail(GBSP_ERR_UNSUPPORTED, "plan sddmm: X and Y must both be BF16 or both E4M3");
    if (X->rows != p->M || Y->rows != p->K || X->cols != Y->cols || X->ld < X->cols || Y->ld < Y->cols)
        return fail(GBSP_ERR_INVALID_ARG, "plan sddmm: shape mismatch");
    const bool fp8 = X->dtype == GBSP_E4M3;
    if (fp8 && ((X->rows > 0 && !X->row_scale) || (Y->rows > 0 && !Y->row_scale)))
        return fail(GBSP_ERR_INVALID_ARG, "plan sddmm: E4M3 X and Y need row scales");
    const int64_t Kd = X->cols;
    const int es = fp8 ? 1 : 2, V = 16 / es;
    if (Kd % V || X->ld % V || Y->ld % V || !aligned16(X->data) || !aligned16(Y->data) || Kd > 32 * 16)
        return fail(GBSP_ERR_ALIGN, "plan sddmm: Kd and leading dimensions multiples of %d, 16-byte aligned X and "
                                    "Y, Kd <= 512", V);
    const int kb = (int)(Kd * es / 128);
    // the tiles pay when a dense block holds enough stored entries to outweigh gathering all
    // its 8 Y rows (measured crossover between 16 and 27 per block on 16,384^2 at 90%, Kd = 256)
    if (tiles < 0) tiles = p->nwin_tc > 0 && p->dense_nnz >= 24 * p->nblocks;
    if (tiles && p->nwin_tc > 0 && ((Kd * es) % 128 || kb < 1 || kb > 8))
        return fail(GBSP_ERR_UNSUPPORTED, "plan sddmm: tensor-core tiles need Kd a multiple of %d and at most %d",
                    128 / es, 1024 / es);
    if (p->nnz == 0 || Kd == 0) return ok();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st;
    if (!tiles) {  // every entry through the CSR kernels on the plan's copy of the pattern
        SddmmProblem q{};
        q.M = (int32_t)p->M;
        q.N = (int32_t)p->K;
        q.Kd = (int32_t)Kd;
        q.nnz = p->nnz;
        q.rowptr = p->rowptr_full;
        q.colidx = p->colidx_full;
        q.svals = svals;
        q.X = X->data;
        q.ldx = X->ld;
        q.x_scale = static_cast<const float *>(X->row_scale);
        q.Y = Y->data;
        q.ldy = Y->ld;
        q.y_scale = static_cast<const float *>(Y->row_scale);
        q.out = out;
        q.dtype = X->dtype;
        const int variant = p->nnz < 32 * p->M ? GBSP_VARIANT_ENTRY : GBSP_VARIANT_ROWSPLIT;
        return (st = launch_sddmm(q, variant, 0, s)) ? st : ok();
    }
    if (p->res_nnz > 0) {  // residual entries through the row-split kernel, at their own positions
        SddmmProblem q{};
        q.M = (int32_t)p->M;
        q.N = (int32_t)p->K;
        q.Kd = (int32_t)Kd;
        q.nnz = p->res_nnz;
        q.rowptr = p->res_rowptr;
        q.colidx = p->res_colidx;
        q.svals = svals;
        q.X = X->data;
        q.ldx = X->ld;
        q.x_scale = static_cast<const float *>(X->row_scale);
        q.Y = Y->data;
        q.ldy = Y->ld;
        q.y_scale = static_cast<const float *>(Y->row_scale);
        q.out = out;
        q.dtype = X->dtype;
        q.pos = p->res_pos;
        if ((st = launch_sddmm(q, GBSP_VARIANT_ROWSPLIT, 0, s))) return st;
    }
    if (p->nwin_tc == 0) return ok();
    CUtensorMap my, mx;
    // copy units of one K-block (16 KB): two unit slots leave room for 5-6 CTAs per SM (two
    // K-blocks per unit, 3 CTAs per SM, measured 1.6x slower for E4M3 at Kd = 256)
    const int kh = 1;
    if ((st = encode_atom_view(Y, fp8, kb, kBC, kh, &my)) || (st = encode_atom_view(X, fp8, kb, kBR, kb, &mx)))
        return st;
    TcSddmmArgs args{p->tc_row0, p->tc_blk, p->blk_col, p->bstart, p->bmask, svals, out,
                     static_cast<const float *>(X->row_scale), static_cast<const float *>(Y->row_scale),
                     (int)p->M, (int)p->K, kb, kh, p->err};
    st = fp8 ? launch_tc_sddmm<true>(my, mx, args, p->nwin_tc, s) : launch_tc_sddmm<false>(my, mx, args, p->nwin_tc, s);
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_plan_info(const gbsp_plan *p, int64_t *info, int n) {
    if (!p || !info || n < 5) return fail(GBSP_ERR_INVALID_ARG, "plan info: need room for 5 values");
    info[0] = p->nwin_tc;
    info[1] = p->nblocks;
    info[2] = p->dense_nnz;
    info[3] = p->res_nnz;
    info[4] = p->threshold;
    return ok();
}

GBSP_EXPORT int gbsp_plan_check(const gbsp_plan *p, void *stream) {
    if (!p) return fail(GBSP_ERR_INVALID_ARG, "plan check: null plan");
    int h = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return check_launch("plan check");
    if (h) {
        cudaMemsetAsync(p->err, 0, sizeof(int), s);  // report each timeout once
        cudaStreamSynchronize(s);
        return fail(GBSP_ERR_TIMEOUT, "a tensor-core window gave up waiting (code %d)", h);
    }
    return ok();
}

GBSP_EXPORT int gbsp_plan_test_withhold(gbsp_plan *p, int32_t chunk) {
    if (!p) return fail(GBSP_ERR_INVALID_ARG, "plan test: null plan");
    p->withhold = chunk;
    return ok();
}

GBSP_EXPORT void gbsp_plan_destroy(gbsp_plan *p) { plan_free(p); }

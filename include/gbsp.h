/*
 * gbsp.h -- C ABI of the GB300 (sm_103a) sparse-matrix library: CSR SpMM and SDDMM.
 *
 * The two operations are the paper's problem statements (Section II-A):
 *   SpMM  (Eq. 1):  C = A B,  A sparse M x K in CSR, B dense K x N, C dense M x N.
 *   SDDMM (Eq. 2):  out = S o (X Y^T) sampled on the pattern of S, i.e. for every stored
 *                   entry p = (i, j) of S:  out[p] = S_ij * <X_i, Y_j>,
 *                   with X dense M x Kd and Y dense N x Kd.
 * The paper writes SpMM as Y = A X with A K x N and X N x D, and SDDMM as
 * Y = A o (B C) with B N x D and C D x N; here the sparse operand is A (or S), the dense
 * feature width is N (SpMM) or Kd (SDDMM), and Y is stored row-major as the transpose of
 * the paper's C so that every gathered row is contiguous.
 *
 * Conventions for every entry point
 *   - All array arguments are DEVICE pointers unless a parameter says "host".  The caller
 *     owns all memory; the library never frees caller memory.
 *   - Dense operands are row-major with a leading dimension ld >= cols (in elements).
 *   - CSR: rowptr is int32[rows + 1] with rowptr[0] = 0 and rowptr[rows] = nnz; colidx is
 *     int32[nnz].  Column indices need not be sorted; repeated indices are summed by SpMM
 *     and computed entry by entry by SDDMM.  rows, cols, N, Kd and nnz must be < 2^31.
 *   - SpMM overwrites C (no accumulation).  SDDMM writes out[] in the CSR order of S.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  Argument errors are returned synchronously and launch
 *     nothing; a failed launch returns GBSP_ERR_CUDA.  Kernel faults surface at the next
 *     synchronisation, as for any CUDA call.
 *   - Inputs are not checked for CSR validity unless opts->validate is set (which costs a
 *     synchronisation); gbsp_csr_validate is the standalone check.  Out-of-range column
 *     indices in an unchecked call are undefined behaviour.
 *   - Results are deterministic: no floating-point atomics; a given variant, launch shape
 *     and input always produce the same bits.
 *   - The entry points are thread-safe; the last-error message is per host thread.
 */
#ifndef GBSP_H
#define GBSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBSP_OK = 0,
    GBSP_ERR_INVALID_ARG = -1, /* null pointer, negative size, ld < cols, dtype mismatch */
    GBSP_ERR_INVALID_CSR = -2, /* validation found a malformed CSR */
    GBSP_ERR_ALIGN = -3,       /* a vectorised variant was forced on unaligned operands */
    GBSP_ERR_UNSUPPORTED = -4, /* a combination the library does not implement */
    GBSP_ERR_CUDA = -5,        /* a CUDA runtime call or launch failed */
    GBSP_ERR_OOM = -6,         /* library workspace could not be allocated */
    GBSP_ERR_TIMEOUT = -7      /* a bounded device-side wait gave up */
} gbsp_status;

typedef enum {
    GBSP_F32 = 0,  /* IEEE binary32 */
    GBSP_BF16 = 1, /* bfloat16, stored as uint16 bits */
    GBSP_E4M3 = 2  /* FP8 E4M3 (OCP), stored as uint8 codes, with one FP32 scale per row */
} gbsp_dtype;

/* Kernel variants of SpMM / SDDMM.  AUTO lets the library choose (see spmm_csr_ex and
 * sddmm_csr_ex for how). */
typedef enum {
    GBSP_VARIANT_AUTO = 0,
    GBSP_VARIANT_ROWSPLIT = 1, /* one warp per row, vectorised gathers */
    GBSP_VARIANT_MERGE = 2,    /* nnz-balanced merge-path split with a carry fix-up pass */
    GBSP_VARIANT_SCALAR = 3,   /* unvectorised, any width / alignment */
    GBSP_VARIANT_ENTRY = 4,    /* SDDMM only: stored entries split evenly across warps regardless of
                                  rows (short or skewed rows); GBSP_ERR_UNSUPPORTED for SpMM */
    GBSP_VARIANT_ROWGROUP = 5, /* SpMM only: several consecutive rows per warp, one lane group each
                                  (rows of a few entries); GBSP_ERR_UNSUPPORTED for SDDMM */
    GBSP_VARIANT_HSP_PLAN = 6, /* a selector label only: the hyper-sparse plan (gbsp_hsp_plan_*);
                                  spmm_csr_ex returns GBSP_ERR_UNSUPPORTED for it */
    GBSP_VARIANT_SELL_PLAN = 7 /* a selector label only: the SELL-C-sigma plan (gbsp_sell_plan_*);
                                  spmm_csr_ex returns GBSP_ERR_UNSUPPORTED for it */
} gbsp_variant;

/* A sparse matrix in CSR form (all pointers device). */
typedef struct {
    int64_t rows, cols, nnz;
    const int32_t *rowptr;   /* int32[rows + 1] */
    const int32_t *colidx;   /* int32[nnz] */
    const void *vals;        /* nnz values of type dtype */
    const float *row_scale;  /* E4M3 only: float[rows], value = row_scale[i] * code; else NULL */
    int32_t dtype;           /* gbsp_dtype */
} gbsp_csr;

/* A dense row-major matrix (data device). */
typedef struct {
    void *data;
    int64_t rows, cols, ld;  /* ld in elements, >= cols */
    const float *row_scale;  /* E4M3 only: float[rows]; else NULL */
    int32_t dtype;           /* gbsp_dtype */
} gbsp_dense;

/* Per-call options; a NULL pointer means all defaults (zero-initialised struct). */
typedef struct {
    int32_t variant;   /* gbsp_variant */
    int32_t validate;  /* nonzero: run gbsp_csr_validate first (synchronises the stream) */
    int32_t unroll;    /* 0 = default; else gathers in flight per lane (1, 2, 4 or 8) */
    int32_t ctas_per_sm; /* merge-path grid: CTAs per SM (0 = default) */
    int32_t vecs;      /* 0 = default; else 16-byte vectors each lane moves per row (1, 2 or 4) */
} gbsp_opts;

/* ---- plain FP32 forms (pointer-and-size signatures), legacy default stream ------------ */

/* SpMM, Eq. 1: C[i, :] = sum over p in row i of vals[p] * B[colidx[p], :].
 * rowptr int32[M+1], colidx int32[nnz], vals float[nnz], B float[K x N] (ld = N),
 * C float[M x N] (ld = N, overwritten).  Returns a gbsp_status. */
int spmm_csr(const int32_t *rowptr, const int32_t *colidx, const float *vals, const float *B,
             float *C, int64_t M, int64_t K, int64_t N);

/* SDDMM, Eq. 2: out[p] = svals[p] * <X[i, :], Y[colidx[p], :]> for every p in row i.
 * rowptr int32[M+1], colidx int32[nnz], svals float[nnz], X float[M x Kd] (ld = Kd),
 * Y float[N x Kd] (ld = Kd), out float[nnz] (overwritten).  Returns a gbsp_status. */
int sddmm_csr(const int32_t *rowptr, const int32_t *colidx, const float *svals, const float *X,
              const float *Y, float *out, int64_t M, int64_t N, int64_t Kd);

/* ---- general forms ----------------------------------------------------------------- */

/* SpMM (Eq. 1) with dtype, leading dimensions, variant and stream.
 * Supported dtype pairs (A, B) -> C: (F32, F32) -> F32, (BF16, BF16) -> F32 and
 * (E4M3, E4M3) -> F32 with per-row scales on both A (s_i) and B (t_k):
 *   C[i, n] = s_i * sum_p qa_p * t_{colidx[p]} * qb[colidx[p], n].
 * Accumulation is FP32 in every form.  B->rows must equal A->cols, C is A->rows x B->cols.
 * GBSP_VARIANT_AUTO balances the work by the pattern's row lengths (load balancing across
 * uneven rows, Section II-D): rows averaging under 12 entries with none past 128 take the
 * row groups, skewed rows (coefficient of variation above 1, or a longest row past 16
 * times the mean and past 256) the merge path, even rows gathered from a B of more than
 * 192 MB (past L2) in rows of at least 256 bytes the row groups, even 128-byte rows from a B
 * of more than 96 MB the merge path, the rest the row split; unvectorisable operands take
 * the scalar kernel.  The row statistics come from one integer pass over
 * rowptr.  The first AUTO call on a pattern measures it and waits for the result (a
 * synchronisation); the choice is kept per (device, rowptr, colidx, rows, cols) for the
 * process (64 patterns, oldest dropped first).  Each later call uses the kept choice and
 * queues one more pass (one small kernel on the stream that writes its counters straight
 * into mapped pinned memory, no wait; at most one in flight per pattern); a later call
 * adopts its result once it has arrived, so another pattern placed at
 * the same addresses gets its own choice from its second call on.  A stale choice costs
 * speed, never correctness.  Under stream capture nothing is queued: a kept choice is used,
 * else the row split.  gbsp_auto_choice reports the choice; gbsp_auto_forget drops them. */
int spmm_csr_ex(const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, const gbsp_opts *opts,
                void *stream);

/* SDDMM (Eq. 2) with dtype, leading dimensions and stream.
 * Supported (S, X, Y): all F32; S F32 with X, Y BF16; S F32 with X, Y E4M3 (per-row
 * scales u_i on X and v_j on Y: out[p] = s_p * u_i * v_j * <qx_i, qy_j>).
 * out is float[S->nnz] in CSR order.  X->rows = S->rows, Y->rows = S->cols,
 * X->cols = Y->cols = Kd.  GBSP_VARIANT_AUTO takes the entry split when rows average under 32
 * stored entries, the merge path on skewed rows (coefficient of variation above 1, or a
 * longest row past 16 times the mean and past 256) and the row split otherwise, from the
 * same kept row statistics as spmm_csr_ex's AUTO (measured, kept and re-measured as
 * described there); unvectorisable operands take the scalar kernel. */
int sddmm_csr_ex(const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y, float *out,
                 const gbsp_opts *opts, void *stream);

/* The split GBSP_VARIANT_AUTO takes on A's pattern (vectorisable operands) for op 0, SpMM
 * (GBSP_VARIANT_ROWSPLIT, _MERGE or _ROWGROUP), or op 1, SDDMM (GBSP_VARIANT_ROWSPLIT, _MERGE
 * or _ENTRY), with a gathered dense operand (B, or Y) of b_bytes bytes in rows of row_bytes
 * bytes (0 and 0 when unknown), written to *variant (host); GBSP_ERR_INVALID_ARG for another
 * op.  stats (host, may be NULL)
 * receives the statistics behind it: {rows, stored entries, sum of squared row lengths,
 * longest row, empty rows}, or -1s for an unmeasured pattern under stream capture.  It is
 * an AUTO call without the product: a new pattern is measured at once (synchronises the
 * stream), a kept one answers from its kept choice and queues a re-measurement.  Only
 * rowptr of A is read. */
int gbsp_auto_choice(const gbsp_csr *A, int32_t op, int64_t b_bytes, int64_t row_bytes, void *stream,
                     int32_t *variant, int64_t *stats);
/* Drops every choice GBSP_VARIANT_AUTO has kept (the next AUTO call measures again). */
void gbsp_auto_forget(void);

/* Checks a CSR on the device: rowptr[0] = 0, rowptr non-decreasing, rowptr[rows] = nnz,
 * 0 <= colidx < cols.  Writes the number of violations to *n_bad (host pointer) and
 * returns GBSP_OK if it is zero, GBSP_ERR_INVALID_CSR otherwise.  Synchronises stream. */
int gbsp_csr_validate(const gbsp_csr *A, void *stream, int64_t *n_bad);

/* ---- precision conversion (the roundings of the BF16 / E4M3 forms) -------------------- */

/* out[i] = bfloat16 round-to-nearest-even of x[i]; n elements (x float, out uint16). */
int gbsp_quantize_bf16(const float *x, uint16_t *out, int64_t n, void *stream);

/* Per-row scaled E4M3: for each row r, scale[r] = max|x| / 448 in FP32 (1 for an all-zero
 * or empty row) and q = E4M3 round-to-nearest-even, saturating, of x / scale[r] (FP32
 * division).  Rows are CSR segments when rowptr (device, int32[nrows+1]) is non-NULL,
 * otherwise nrows dense rows of ncols entries with leading dimension ld (q uses ld too). */
int gbsp_quantize_e4m3_rows(const float *x, const int32_t *rowptr, int64_t nrows, int64_t ncols,
                            int64_t ld, uint8_t *q, float *scale, void *stream);

/* ---- host-resident operands, streamed in row chunks ----------------------------------------- */

/* SpMM (Eq. 1, when B, C and N > 0 are given) and / or SDDMM (Eq. 2, when X, Y, out and
 * Kd > 0 are given) on FP32 operands in HOST memory (pinned memory lets the copies overlap
 * the kernels): rowptr[M+1], colidx[nnz], vals[nnz] (also the S values of SDDMM), B[K x N],
 * C[M x N], X[M x Kd], Y[K x Kd], out[nnz], all row-major with ld = width.  The library
 * copies B, X, Y once, then streams the matrix in `chunks` row chunks of about equal
 * entries (default 8 when < 1) through `slots` device buffers (default 2 when < 2) on its
 * own copy-in, compute and copy-out streams, so chunk i+1 arrives while chunk i computes and
 * chunk i-1's results return.  Device workspace comes from the library's pool.  The call
 * returns once everything is queued; `stream` (the caller's) waits for the last result, so
 * synchronise it before reading C and out.  N and Kd must be multiples of 4. */
int gbsp_spmm_sddmm_host(const int32_t *rowptr, const int32_t *colidx, const float *vals, const float *B,
                         float *C, int64_t N, const float *X, const float *Y, float *out, int64_t Kd, int64_t M,
                         int64_t K, int64_t nnz, int32_t chunks, int32_t slots, void *stream);

/* ---- condensed-tile tensor-core plan (BF16, E4M3) ----------------------------------------- */

/* A plan splits a BF16 or per-row-scaled E4M3 CSR matrix A into dense 16 x 8 blocks
 * (aligned; at least `threshold` stored entries; when threshold < 1, 14 for BF16 and 10 for
 * E4M3) and a residual CSR.  Executing it computes C = A B (Eq. 1) as: residual SpMM through the CSR
 * kernels (which writes C), then, for each 16-row window holding dense blocks, a tcgen05 MMA
 * of the window's condensed 16 x Kc tile with the Kc gathered rows of B (FP32 accumulation
 * in tensor memory), added into C.  The plan keeps its own device copy of everything it
 * needs; A (and its row scales) may be freed after creation.
 * BF16 (kind::f16): A->dtype BF16; at execution B BF16 (K x N).
 * E4M3 (kind::f8f6f4): A->dtype E4M3 with A->row_scale (M floats, value = s_i * q);
 * at execution B E4M3 with B->row_scale (K floats, value = t_k * q).  A scale along the
 * contraction cannot be applied after the MMA, so each execution first folds t into the
 * dense-block values, a~_ik = (s_i q_ik) t_k in FP32, and requantises every window row to
 * E4M3 with a power-of-two scale u_r (the smallest with max |a~| <= 448 u_r, at least
 * 2^-126); the epilogue multiplies the row's MMA result by u_r.  The residual uses s and t
 * as given.  An E4M3 plan's executions rewrite its tiles: order them on one stream.
 * Both: strictly increasing column indices in every row (GBSP_ERR_UNSUPPORTED otherwise);
 * C FP32 (M x N); when any window is dense, 64 <= N <= 512, N and B->ld multiples of 16
 * bytes' worth of elements (8 BF16, 16 E4M3) and B 16-byte aligned.
 * residual_opts (may be NULL) chooses the residual kernel.  gbsp_plan_create synchronises
 * the stream; gbsp_plan_execute is asynchronous and may be repeated with new B and C.
 * Device-side waits in the tensor-core kernel give up after about a second and record it;
 * gbsp_plan_check (synchronous) returns GBSP_ERR_TIMEOUT if any did since the last check.
 * gbsp_plan_info fills info[0..4] = {dense windows, dense blocks (padded per window to a
 * pipeline stage: 8 BF16 or 16 E4M3 blocks), entries inside dense blocks, residual
 * entries, threshold}. */
typedef struct gbsp_plan gbsp_plan;
int gbsp_plan_create(const gbsp_csr *A, int32_t threshold, const gbsp_opts *residual_opts, void *stream,
                     gbsp_plan **out);
int gbsp_plan_execute(const gbsp_plan *plan, const gbsp_dense *B, gbsp_dense *C, void *stream);
/* SDDMM on the plan's sparsity pattern (Eq. 2): out[p] = svals[p] * <X_i, Y_j> for every
 * stored entry p = (i, j) of the matrix the plan was made from, in that matrix's CSR order
 * (svals and out: device float[nnz]; the plan's own values are not used).  X (M x Kd) and
 * Y (K x Kd) both BF16, or both E4M3 with row scales (X->row_scale u_i, Y->row_scale v_j;
 * the result is scaled by u_i v_j).  Residual entries run on the row-split CSR kernel; the
 * 16 x 8 outputs of each dense block come from one tcgen05 MMA per 16 blocks and K-step:
 * D (128 x 16) = Y_g X_w^T with the blocks' Y rows and the window's X rows in shared
 * memory (TMA), FP32 accumulation in tensor memory, and the epilogue writes the stored
 * entries only.  Requirements: Kd and both leading dimensions multiples of 16 bytes' worth
 * of elements, 16-byte aligned X and Y, Kd <= 512 (GBSP_ERR_ALIGN otherwise); when any
 * window is dense and the tiles are used, Kd a multiple of 64 (BF16) or 128 (E4M3)
 * (GBSP_ERR_UNSUPPORTED).  tiles: 1 uses the tiles as above, 0 runs every entry through the
 * CSR kernels on the plan's copy of the pattern, < 0 chooses: the tiles when the dense
 * blocks average at least 24 stored entries (below that, gathering a block's 8 Y rows costs
 * more than its entries' rows).  Asynchronous; waits are bounded as in gbsp_plan_execute
 * (see gbsp_plan_check). */
int gbsp_plan_sddmm(const gbsp_plan *plan, const float *svals, const gbsp_dense *X, const gbsp_dense *Y, float *out,
                    int32_t tiles, void *stream);
int gbsp_plan_info(const gbsp_plan *plan, int64_t *info, int n);
int gbsp_plan_check(const gbsp_plan *plan, void *stream);
/* Testing the timeout path (no counterpart in the paper): while chunk >= 0, the first
 * dense window's kernel never loads that stage, so its MMA warp's wait runs out after about
 * a second, the kernel records it and returns; gbsp_plan_check then reports
 * GBSP_ERR_TIMEOUT (once) and the context stays usable.  chunk = -1 switches it off. */
int gbsp_plan_test_withhold(gbsp_plan *plan, int32_t chunk);
void gbsp_plan_destroy(gbsp_plan *plan);

/* ---- grouped SpMM / SDDMM over many problems (persistent launches in one CUDA graph) ------- */

/* G independent problems (arrays of G host-side descriptors, device data) of uneven size in
 * one graph: SpMM C_g = A_g B_g (Eq. 1) with A_g and B_g both FP32 or both BF16 and C_g FP32,
 * widths and leading dimensions multiples of 16 bytes, rows 16-byte aligned; or SDDMM
 * out_g = S_g o (X_g Y_g^T) (Eq. 2) with FP32 S_g values, X_g, Y_g both FP32 or both BF16,
 * Kd <= 256 (FP32) / 512 (BF16), out[g] device float[nnz_g].  All problems of a batch share
 * the dense dtype.  The plan reads each rowptr to the host (synchronises the stream), builds
 * tiles of consecutive rows with about 512 entries, groups them by the lane layout their
 * problem's width needs, and records the ticket resets plus one persistent launch per
 * layout in use (at most 3 for SpMM, 5 for SDDMM) into a CUDA graph that
 * gbsp_batch_plan_execute replays (asynchronous); SDDMM tiles of short rows (under 32
 * entries on average) run the entry split (GBSP_VARIANT_ENTRY);
 * the plan keeps the caller's pointers.  spmm_csr_batched / sddmm_csr_batched are the
 * one-shot forms (create, execute, synchronise, destroy). */
typedef struct gbsp_batch_plan gbsp_batch_plan;
int gbsp_batch_plan_create_spmm(int G, const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, void *stream,
                                gbsp_batch_plan **out);
int gbsp_batch_plan_create_sddmm(int G, const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y,
                                 float *const *out, void *stream, gbsp_batch_plan **plan);
int gbsp_batch_plan_execute(const gbsp_batch_plan *plan, void *stream);
void gbsp_batch_plan_destroy(gbsp_batch_plan *plan);
int spmm_csr_batched(int G, const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, void *stream);
int sddmm_csr_batched(int G, const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y, float *const *out,
                      void *stream);

/* ---- batched graph chain (one persistent launch in a CUDA graph) ---------------------------- */

/* For each graph g of a batch of G (arrays of G host-side descriptors, device data):
 *   E_g = S_g o (H_g H_g^T) on the pattern of S_g      (Eq. 2 with X = Y = H_g)
 *   O_g = E_g H_g                                       (Eq. 1 with the values E_g)
 * S_g: square FP32 CSR with nnz given; H_g, O_g: BF16 n_g x N_g (N_g a multiple of 8,
 * at most 256, rows 16-byte aligned); E[g]: device float[nnz_g] in CSR order.  Accumulation
 * is FP32; O is rounded to BF16 (nearest even).  The plan builds a device work list of row
 * tiles (about edges_per_tile edges each, default 512 when <= 0) over all graphs and
 * records one persistent launch, which takes tiles from an atomic ticket, into a CUDA
 * graph; gbsp_gnn_plan_execute replays it on the stream (asynchronous).  The plan keeps the
 * caller's pointers: the data may change between executions, the allocations may not.
 * gbsp_gnn_plan_create reads every rowptr to the host (synchronises the stream).
 * gbsp_gnn_plan_info fills {graphs, tiles, rows, edges}.  gnn_sddmm_spmm_batched is the
 * one-shot form (create, execute, synchronise, destroy). */
typedef struct gbsp_gnn_plan gbsp_gnn_plan;
int gbsp_gnn_plan_create(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O,
                         int32_t edges_per_tile, void *stream, gbsp_gnn_plan **out);
/* GAT-style form (flags GBSP_GNN_SOFTMAX; the attention layer the paper names as the
 * SDDMM -> SpMM use case): between the two products each row's scores are normalised,
 *   alpha_ij = exp(E_ij - m_i) / sum_j exp(E_ij - m_i),  m_i = max_j E_ij  (stored entries),
 * O_g = alpha H_g, and E[g] receives alpha.  The kernel keeps, per lane group, a running
 * sum and accumulator against a reference score (online softmax) and merges the groups at
 * each row's end; the exponentials are exp2f of base-2 scaled scores.  Rows without entries
 * give zero O rows.  gbsp_gnn_plan_create is the
 * flags = 0 form; gnn_gat_batched the one-shot softmax form. */
#define GBSP_GNN_SOFTMAX 1
int gbsp_gnn_plan_create_ex(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O,
                            int32_t edges_per_tile, int32_t flags, void *stream, gbsp_gnn_plan **out);
int gbsp_gnn_plan_execute(const gbsp_gnn_plan *plan, void *stream);
int gbsp_gnn_plan_info(const gbsp_gnn_plan *plan, int64_t *info, int n);
void gbsp_gnn_plan_destroy(gbsp_gnn_plan *plan);
int gnn_sddmm_spmm_batched(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O,
                           void *stream);
int gnn_gat_batched(int G, const gbsp_csr *S, const gbsp_dense *H, float *const *E, gbsp_dense *O, void *stream);

/* ---- K-range-binned SpMM (B larger than L2) ---------------------------------------------- */

/* SpMM, Eq. 1, C = A B for FP32 A (M x K, CSR) and FP32 B (K x N), with A's columns cut into
 * S slices of W consecutive indices (the 1.5D binning of A's nonzeros by K-range, Section
 * II-C and the column-range filter of Section III-A): pass s sums, for every row, the
 * entries whose column lies in slice s, so its B
 * gathers stay inside W rows of B (about 48 MB by default, held in L2).  Pass 0 writes C,
 * later passes add to the rows with entries in their slice.  The result is Eq. 1's sum in
 * slice order (FP32, deterministic).
 *
 * gbsp_kbin_plan_create checks A (gbsp_csr_validate's checks, and column indices
 * non-decreasing within each row: GBSP_ERR_INVALID_CSR otherwise), chooses W (slice_cols, or
 * for slice_cols = 0 the number of B rows of width N that fill 48 MB, at least 1024; capped
 * at K; at most 4096 slices, GBSP_ERR_INVALID_ARG beyond) and stores, for every slice
 * boundary and row, the first entry at or past it ((S + 1) x M int32 on the device).  It
 * synchronises the stream.  The plan keeps A's pointers: the values may change between
 * executions, the pattern and the allocations may not.
 * gbsp_kbin_plan_execute: B float[K x N] (ld >= N), C float[M x N] (ld >= N, overwritten);
 * N and both ld multiples of 4, B and C 16-byte aligned (GBSP_ERR_ALIGN otherwise); any N,
 * not only the one W was sized for.  S launches on the stream (asynchronous); the current
 * device must be the plan's.
 * gbsp_kbin_plan_info fills {slices S, slice width W, rows M, nnz}. */
typedef struct gbsp_kbin_plan gbsp_kbin_plan;
int gbsp_kbin_plan_create(const gbsp_csr *A, int64_t N, int64_t slice_cols, void *stream, gbsp_kbin_plan **out);
int gbsp_kbin_plan_execute(const gbsp_kbin_plan *plan, const gbsp_dense *B, gbsp_dense *C, void *stream);
int gbsp_kbin_plan_info(const gbsp_kbin_plan *plan, int64_t *info, int n);
void gbsp_kbin_plan_destroy(gbsp_kbin_plan *plan);

/* ---- hyper-sparse SpMM (rows binned by length) -------------------------------------------- */

/* SpMM, Eq. 1, C = A B for FP32 A (M x K, CSR) and B (K x N), for matrices whose rows hold
 * a few entries or none (past 99.9% sparsity; the weak spot the paper reports for its own
 * design, Section IV-C, and its future work, Section V).  gbsp_hsp_plan_create checks A as
 * gbsp_csr_validate does (GBSP_ERR_INVALID_CSR), reads the row lengths (synchronises the
 * stream) and bins the rows: long rows (more than 32 entries) take one warp each as in the
 * row split; short rows (1 to 32), sorted by length, take one lane group each (several rows
 * per warp); empty rows get their zero C rows.  The plan keeps A's pointers (values may
 * change between executions; the pattern and allocations may not), the long and empty
 * row lists (int32) and a 16-byte record per short row {row, first entry, end, first
 * column index} on the device.
 * gbsp_hsp_plan_execute: B float[K x N] (ld >= N), C float[M x N] (ld >= N, overwritten);
 * N and both ld multiples of 4, B and C 16-byte aligned (GBSP_ERR_ALIGN otherwise).  One
 * launch on the stream (asynchronous); each row's sum runs in its stored order within a
 * short row, in the row split's order within a long row.
 * gbsp_hsp_plan_info fills {long rows, short rows, empty rows, nnz}. */
typedef struct gbsp_hsp_plan gbsp_hsp_plan;
int gbsp_hsp_plan_create(const gbsp_csr *A, void *stream, gbsp_hsp_plan **out);
int gbsp_hsp_plan_execute(const gbsp_hsp_plan *plan, const gbsp_dense *B, gbsp_dense *C, void *stream);
int gbsp_hsp_plan_info(const gbsp_hsp_plan *plan, int64_t *info, int n);
void gbsp_hsp_plan_destroy(gbsp_hsp_plan *plan);

/* ---- SELL-C-sigma SpMM (sliced, padded, column-major) ------------------------------------ */

/* SpMM, Eq. 1, C = A B for FP32 A (M x K, CSR) and B (K x N), through SELL-C-sigma: the
 * sliced padded format of the paper's SELLPACK-like stream (Section III-A) and of its
 * future work on formats (Section V).  gbsp_sell_plan_create checks A as gbsp_csr_validate
 * does (nnz must be given; GBSP_ERR_INVALID_CSR), reads rowptr to the host (synchronises
 * the stream), sorts the rows by decreasing length within windows of sigma rows (sigma <= 0
 * or > M: one window; else a multiple of C), cuts the sorted rows into slices of C rows
 * (C <= 0: 64; a multiple of 8, at most 1024), pads each slice to its longest row and
 * stores it column-major (entry j of the slice's row r at slot j * C + r) in the plan's own
 * device arrays: the row order and lengths (int32 each per row), the slice offsets (int64)
 * and the slots (int32 column and FP32 value each, padding included).  A may be freed
 * after creation.
 * gbsp_sell_plan_execute: one lane group per row, several rows per warp, every group
 * stopping at its own row's length (padding is never read); B float[K x N] (ld >= N), C
 * float[M x N] (ld >= N, overwritten); N and both ld multiples of 4, B and C 16-byte
 * aligned (GBSP_ERR_ALIGN otherwise); C must be a multiple of 8 x (rows per warp), which
 * holds for the default C = 64 from N = 16 on (GBSP_ERR_UNSUPPORTED otherwise).  One launch,
 * asynchronous; each row's sum runs in its stored order.
 * gbsp_sell_plan_info fills {slices, C, sigma, slots including padding, nnz}. */
typedef struct gbsp_sell_plan gbsp_sell_plan;
int gbsp_sell_plan_create(const gbsp_csr *A, int32_t C, int32_t sigma, void *stream, gbsp_sell_plan **out);
int gbsp_sell_plan_execute(const gbsp_sell_plan *plan, const gbsp_dense *B, gbsp_dense *C, void *stream);
int gbsp_sell_plan_info(const gbsp_sell_plan *plan, int64_t *info, int n);
void gbsp_sell_plan_destroy(gbsp_sell_plan *plan);

/* ---- kernel selection: features, autotuner, MLP ------------------------------------------- */

/* The 24 SpMM variants the selector chooses among, as options for spmm_csr_ex:
 *   0..8   row-split, vecs {1,2,4} x unroll {2,4,8}     (index = 3 * vecs_index + unroll_index)
 *   9..17  merge path, the same nine layouts
 *   18..20 merge path with 1 CTA per SM and vecs {1,2}, or 2 CTAs per SM and vecs 1; unroll 4
 *   21     the SELL-C-sigma plan: out->variant = GBSP_VARIANT_SELL_PLAN, meaning "create a
 *          gbsp_sell_plan of A once (C = 64, one sort window) and execute it" (FP32 only)
 *   22     row groups (GBSP_VARIANT_ROWGROUP), default layout
 *   23     the hyper-sparse plan: out->variant = GBSP_VARIANT_HSP_PLAN, meaning "create a
 *          gbsp_hsp_plan of A once and execute it" (FP32 only); not an spmm_csr_ex option. */
int gbsp_variant_opts(int variant, gbsp_opts *out);
/* The SDDMM variants (Eq. 2) the SDDMM selector chooses among, as options for sddmm_csr_ex:
 * index = 3 * split + vecs_index, split 0 row split, 1 merge path, 2 entry split, vecs
 * {1, 2, 4}; 9 variants (indices 0..8), GBSP_ERR_INVALID_ARG beyond. */
int gbsp_sddmm_variant_opts(int variant, gbsp_opts *out);

/* 16 features of a CSR matrix for a dense width N and dtype, written to feats (device,
 * float[16]) in one pass over rowptr / colidx (asynchronous):
 *   0 log2 M, 1 log2 K, 2 log2(1 + nnz), 3 log2(density), 4 log2(1 + mean row length),
 *   5 log2(1 + row-length standard deviation), 6 its coefficient of variation,
 *   7 log2(1 + max row length), 8 max / mean row length, 9 fraction of empty rows,
 *   10 mean |j - floor(i K / M)| / K, 11 max of the same / K, 12 fraction of consecutive
 *   entries of a row less than 8 columns apart, 13 fraction of entries whose column is also
 *   stored in the next row (rows sorted by column), 14 log2 N, 15 dtype. */
int gbsp_features(const gbsp_csr *A, int64_t N, int32_t dtype, float *feats, void *stream);

/* norm[0..15] = mean, norm[16..31] = standard deviation (1 where 0) of n feature rows. */
int gbsp_feature_norm(const float *feats, int n, float *norm, void *stream);

/* MLP 16 -> 64 -> 64 -> 24 with ReLU on the hidden layers; weights (device, 6,808 floats)
 * laid out W1[64x16], b1[64], W2[64x64], b2[64], W3[24x64], b3[24] (row-major, out x in);
 * inputs standardised with norm.  out (n x 24, may be NULL) receives the predictions, choice
 * (n, may be NULL) the index of the smallest. */
int gbsp_mlp_predict(const float *weights, const float *norm, const float *feats, int n, float *out,
                     int32_t *choice, void *stream);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) of the masked squared
 * error sum(mask (y - target)^2) / sum(mask) over minibatches of `batch` (<= 64) samples
 * taken in turn from order[0..norder) (wrapping); adam holds the first then the second
 * moments (2 x 6,808 floats); t0 = steps already taken.  One CTA, deterministic. */
int gbsp_mlp_train(float *weights, float *adam, const float *norm, const float *feats, const float *targets,
                   const float *mask, const int32_t *order, int norder, int steps, int batch, float lr, int t0,
                   void *stream);

/* Times every SpMM variant of gbsp_variant_opts on A, B, C (one untimed call, then reps
 * timed calls with CUDA events; variants 21 and 23 build a SELL-C-sigma or hyper-sparse
 * plan of A first, outside the timed calls, so A->nnz must be given) and writes times_ms[24] (host; INFINITY where a
 * variant does not apply) and *best (host).  Synchronises the stream; C ends up holding the
 * last variant's result. */
int gbsp_autotune(const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, int reps, float *times_ms,
                  int32_t *best, void *stream);
/* The same for SDDMM: times the 9 variants of gbsp_sddmm_variant_opts on S, X, Y, out and
 * writes times_ms[24] (INFINITY at indices 9..23 and where a variant does not apply) and
 * *best.  Synchronises the stream; out ends up holding the last variant's result. */
int gbsp_autotune_sddmm(const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y, float *out, int reps,
                        float *times_ms, int32_t *best, void *stream);

/* ---- allocation-free variant ---------------------------------------------------------- */

/* The paper has no counterpart of this entry point.  It serves callers that must not
 * allocate device memory during a call: a process whose HBM is already handed out by
 * another allocator (a framework's caching allocator, or a fixed arena in a serving
 * process), where an allocation can fail at call time, and a latency-bound loop that
 * cannot absorb an allocation and the synchronisation it may bring.
 * FP32 SpMM with the meaning of spmm_csr (Eq. 1; rowptr, colidx, vals, B, C device; B and
 * C with ld = N; C overwritten), on the given stream, through the merge-path kernels.
 * Their carry buffers live in one fixed 4 MiB device array owned by the library, which
 * every GPU that loads the library holds until the process exits; nothing is allocated.
 * Limits: N <= 1024 and a multiple of 4, B and C 16-byte aligned; a larger N returns
 * GBSP_ERR_INVALID_ARG, misalignment GBSP_ERR_ALIGN.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the life of the process: make that first call before any stream capture.
 * cudaDeviceReset destroys the array with the device's context and leaves the kept address
 * stale, so do not call this entry point on a device after resetting it.  All calls share
 * the one array, so calls that can overlap on the GPU (unordered streams) race and must be
 * serialised by the caller.  Each call writes every scratch element before reading it, so
 * what a previous call left there does not matter. */
int spmm_csr_noalloc(const int32_t *rowptr, const int32_t *colidx, const float *vals, const float *B,
                     float *C, int64_t M, int64_t K, int64_t N, void *stream);

/* ---- measurement utility (no counterpart in the paper) ------------------------------- */

/* Gather-bandwidth probe: reads the rows table[idx[p]] (row_bytes = 128, 256, 512 or 1024 bytes
 * each, consecutive rows ld_bytes apart) for p in [0, n) with the lane layout of the
 * SpMM / SDDMM kernels (16-byte vectors, several rows in flight per lane, indices loaded
 * coalesced and shuffled to the lane groups) and no arithmetic but an XOR per vector, so
 * n * row_bytes / time is the ceiling of that access pattern (L2 when the table fits in it).
 * table: device, 16-byte aligned, `rows` rows; every idx[p] must be in [0, rows) (not
 * checked on the device).  sink: device, blocks * 256 uint32 (written, meaningless).
 * blocks: grid size (256 threads each); unroll: 4 or 8 rows in flight per lane.
 * Asynchronous on `stream`; GBSP_ERR_UNSUPPORTED for another row_bytes, GBSP_ERR_ALIGN for
 * a misaligned table or ld_bytes. */
int gbsp_gather_probe(const void *table, int64_t rows, int64_t row_bytes, int64_t ld_bytes, const int32_t *idx,
                      int64_t n, uint32_t *sink, int32_t blocks, int32_t unroll, void *stream);

/* ---- errors ------------------------------------------------------------------------ */

const char *gbsp_status_string(int status);
/* Status and message of the last failing call on this host thread (GBSP_OK if none). */
int gbsp_get_last_error(void);
const char *gbsp_last_error_message(void);

/* Number of SMs of the current device as the library sees it (0 on error). */
int gbsp_device_sm_count(void);

/* Number of CUDA kernels this library has launched in the process so far (all threads).
 * Benchmarks difference it around a timed region to count the library's launches. */
int64_t gbsp_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GBSP_H */

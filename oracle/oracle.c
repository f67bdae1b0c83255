/*
 * Plain FP64 CPU oracle for CSR SpMM and SDDMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the library's product path calls, links or loads
 * this file: only the tests, the benchmark's CPU-baseline leg and the smoke check do.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is the plain definition it cites, written as straight loops in double
 * precision with no blocking or reordering; OpenMP only splits independent output rows
 * across threads and never changes the order of any sum.
 *
 * Notation: A (or S) is an M x K (or M x N) CSR matrix with int32 row pointers and column
 * indices; dense operands are row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int pick_threads(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return pick_threads(0); }

/*
 * SpMM, Eq. 1 (Section II-A: Y = A X with A sparse) in this library's naming C = A B:
 *   C[i, n] = sum over p in [rowptr[i], rowptr[i+1]) of vals[p] * B[colidx[p], n]
 * which is the per-nonzero multiply-accumulate of the worker task (Section III-A-1).
 * scale[i, n] = sum of |vals[p]| * |B[colidx[p], n]| (the per-output error scale).
 * Repeated column indices in a row are separate terms of the sum.  C is overwritten.
 * scale may be NULL.
 */
void oracle_spmm_f64(int64_t M, int64_t K, int64_t N, const int32_t *rowptr,
                     const int32_t *colidx, const double *vals, const double *B, double *C,
                     double *scale, int nthreads) {
    (void)K;
    int nt = pick_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < M; ++i) {
        double *c = C + i * N;
        double *s = scale ? scale + i * N : 0;
        for (int64_t n = 0; n < N; ++n) {
            c[n] = 0.0;
            if (s) s[n] = 0.0;
        }
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double a = vals[p];
            const double *b = B + (int64_t)colidx[p] * N;
            for (int64_t n = 0; n < N; ++n) {
                c[n] += a * b[n];
                if (s) s[n] += fabs(a) * fabs(b[n]);
            }
        }
    }
}

/*
 * SDDMM, Eq. 2 (Section II-A: Y = A o (B C), computed only where A is nonzero,
 * Section III-B) in this library's naming, with Y here the N x Kd row-major transpose of
 * the paper's C:
 *   out[p] = svals[p] * sum over k of X[i, k] * Y[colidx[p], k]   for p in row i
 * scale[p] = |svals[p]| * sum over k of |X[i, k]| * |Y[colidx[p], k]|.
 * out is in the CSR order of S.  scale may be NULL.
 */
void oracle_sddmm_f64(int64_t M, int64_t N, int64_t Kd, const int32_t *rowptr,
                      const int32_t *colidx, const double *svals, const double *X,
                      const double *Y, double *out, double *scale, int nthreads) {
    (void)N;
    int nt = pick_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < M; ++i) {
        const double *x = X + i * Kd;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double *y = Y + (int64_t)colidx[p] * Kd;
            double dot = 0.0, adot = 0.0;
            for (int64_t k = 0; k < Kd; ++k) {
                dot += x[k] * y[k];
                adot += fabs(x[k]) * fabs(y[k]);
            }
            out[p] = svals[p] * dot;
            if (scale) scale[p] = fabs(svals[p]) * adot;
        }
    }
}

/* ---- BF16: 1 sign bit, 8 exponent bits, 7 stored significand bits -------------------- */

/*
 * Round an FP32 value to the nearest BF16 value, ties to even, returning its bits.
 * BF16 keeps the upper 16 bits of the FP32 encoding, so the discarded low half decides
 * the rounding: above half an ulp rounds up, below rounds down, exactly half rounds to
 * the even kept pattern.  NaN stays a quiet NaN.
 */
static uint16_t bf16_rne(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu))
        return (uint16_t)((u >> 16) | 0x0040u);
    uint32_t hi = u >> 16, lo = u & 0xffffu;
    if (lo > 0x8000u || (lo == 0x8000u && (hi & 1u))) hi += 1u;
    return (uint16_t)hi;
}

void oracle_bf16_round(int64_t n, const float *x, uint16_t *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = bf16_rne(x[i]);
}

void oracle_bf16_decode(int64_t n, const uint16_t *h, double *out) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = (uint32_t)h[i] << 16;
        float f;
        memcpy(&f, &u, 4);
        out[i] = (double)f;
    }
}

/* ---- FP8 E4M3 (OCP): 1 sign, 4 exponent bits (bias 7), 3 significand bits ------------
 * Normal values (1 + m/8) * 2^(e-7) for e in 1..15 (e = 15 with m = 7 is NaN), so the
 * largest finite value is 1.75 * 2^8 = 448; subnormals m * 2^-9; no infinities. */

/* Value of an E4M3 code. */
static double e4m3_value(uint8_t q) {
    int s = q >> 7, e = (q >> 3) & 15, m = q & 7;
    double v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0)
        v = ldexp((double)m, -9);
    else
        v = ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

void oracle_e4m3_decode(int64_t n, const uint8_t *q, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_value(q[i]);
}

/* Nearest E4M3 value, ties to even, magnitudes past the largest finite value clamped to
 * it (saturating conversion).  Every step below is exact in double. */
static uint8_t e4m3_rne_sat(float xf) {
    double x = (double)xf;
    uint8_t sign = signbit(x) ? 0x80 : 0x00;
    double a = fabs(x);
    if (isnan(x)) return (uint8_t)(sign | 0x7f);
    if (a >= 448.0) return (uint8_t)(sign | 0x7e);
    if (a < ldexp(1.0, -6)) {              /* subnormal range: multiples of 2^-9 */
        double m = nearbyint(ldexp(a, 9)); /* default rounding mode: ties to even */
        return (uint8_t)(sign | (uint8_t)m); /* m == 8 is the smallest normal, code 0x08 */
    }
    int e2;
    frexp(a, &e2); /* a = f * 2^e2 with f in [0.5, 1) */
    int e = e2 - 1; /* a in [2^e, 2^(e+1)) */
    double m = nearbyint(ldexp(a, 3 - e) - 8.0); /* 3 significand bits, ties to even */
    if (m == 8.0) {
        m = 0.0;
        e += 1;
    }
    return (uint8_t)(sign | (uint8_t)((e + 7) << 3) | (uint8_t)m);
}

void oracle_e4m3_round(int64_t n, const float *x, uint8_t *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_rne_sat(x[i]);
}

/*
 * Per-row scaled E4M3 quantisation: row r's scale is s_r = max |x| / 448 computed in FP32
 * (1 for a row that is all zero or empty), and each entry is stored as the E4M3 rounding
 * of the FP32 quotient x / s_r.  Rows are CSR segments when rowptr is given, otherwise
 * consecutive runs of ncols entries.
 */
void oracle_e4m3_rows(int64_t nrows, const int32_t *rowptr, int64_t ncols, const float *x,
                      uint8_t *q, float *scale) {
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t b = rowptr ? rowptr[r] : r * ncols;
        int64_t e = rowptr ? rowptr[r + 1] : (r + 1) * ncols;
        float amax = 0.0f;
        for (int64_t p = b; p < e; ++p) {
            float v = fabsf(x[p]);
            if (v > amax) amax = v;
        }
        volatile float s = amax / 448.0f; /* FP32 division, as the format definition */
        if (amax == 0.0f) s = 1.0f;
        scale[r] = s;
        for (int64_t p = b; p < e; ++p) {
            volatile float t = x[p] / s;
            q[p] = e4m3_rne_sat(t);
        }
    }
}

/*
 * Operands of the E4M3 condensed-tile SpMM (the library's reading of how per-row scales of
 * B, which lie along the contraction of Eq. 1, reach tensor-core tiles; the paper itself
 * has no tensor-core or FP8 design).  A is an M x K CSR matrix of E4M3 codes qa with row
 * scales sa (value s_i * dec(q)); tb holds B's row scales t_k.
 *   1. Blocks: A is cut into aligned blocks of 16 rows x 8 columns; a block whose stored
 *      entries number at least `threshold` (10 when threshold < 1) is dense.
 *   2. Fold: every entry of a dense block takes a~ = fl32(fl32(s_i * dec(q)) * t_k).
 *   3. Row scale: for each row i, amax = max |a~| over the row's dense-block entries and
 *      u_i = 2^e with e the smallest integer >= -126 such that amax <= 448 * 2^e.
 *   4. Requantise: q'_ik = E4M3 (nearest, ties to even, saturating) of a~ / u_i.
 *   5. The tensor cores then multiply u_i * dec(q'_ik); residual entries (outside dense
 *      blocks) keep s_i * dec(q_ik) * t_k.
 * Outputs per entry: codes (q' for dense entries, q otherwise), dense (1 / 0), eff (the
 * FP64 value the product uses: u_i dec(q') or s_i dec(q) t_k, the latter exact in double);
 * per row: exp_out (e; -126 for a row without dense entries).  Any output may be NULL.
 */
void oracle_e4m3_fold(int64_t M, int64_t K, const int32_t *rowptr, const int32_t *colidx,
                      const uint8_t *qa, const float *sa, const float *tb, int threshold,
                      uint8_t *codes, uint8_t *dense, double *eff, int32_t *exp_out) {
    const int64_t bcols = (K + 7) / 8;
    const int64_t nwin = (M + 15) / 16;
    const int thr = threshold >= 1 ? threshold : 10;
    /* step 1: stored entries per block, one window (16 rows) at a time */
    int64_t *count = (int64_t *)calloc((size_t)(bcols > 0 ? bcols : 1), sizeof(int64_t));
    for (int64_t w = 0; w < nwin; ++w) {
        const int64_t r0 = 16 * w, r1 = r0 + 16 < M ? r0 + 16 : M;
        for (int64_t b = 0; b < bcols; ++b) count[b] = 0;
        for (int64_t i = r0; i < r1; ++i)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) count[colidx[p] / 8] += 1;
        for (int64_t i = r0; i < r1; ++i) {
            /* steps 2 and 3: fold the row's dense entries and find its exponent */
            float amax = 0.0f;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int is_dense = count[colidx[p] / 8] >= thr;
                if (dense) dense[p] = (uint8_t)is_dense;
                if (is_dense) {
                    volatile float sq = sa[i] * (float)e4m3_value(qa[p]);
                    volatile float at = sq * tb[colidx[p]];
                    if (fabsf(at) > amax) amax = fabsf(at);
                }
            }
            int e = -126;
            while ((double)amax > ldexp(448.0, e)) ++e;
            if (exp_out) exp_out[i] = e;
            /* steps 4 and 5 */
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int is_dense = count[colidx[p] / 8] >= thr;
                if (is_dense) {
                    volatile float sq = sa[i] * (float)e4m3_value(qa[p]);
                    volatile float at = sq * tb[colidx[p]];
                    const uint8_t q2 = e4m3_rne_sat((float)ldexp((double)at, -e));
                    if (codes) codes[p] = q2;
                    if (eff) eff[p] = ldexp(e4m3_value(q2), e);
                } else {
                    if (codes) codes[p] = qa[p];
                    if (eff) eff[p] = (double)sa[i] * e4m3_value(qa[p]) * (double)tb[colidx[p]];
                }
            }
        }
    }
    free(count);
}

// Kernel selection: matrix features, the exhaustive autotuner, and a small MLP (16 -> 64
// -> 64 -> 24, ReLU) that predicts each SpMM variant's time relative to the best, trained
// and evaluated by hand-written kernels.
#include <math.h>

#include "common.cuh"

namespace gbsp {
namespace sel {

constexpr int kF = 16, kH = 64, kV = 24;
constexpr int kSddmmVariants = 9;
constexpr int kW1 = kH * kF, kB1 = kH, kW2 = kH * kH, kB2 = kH, kW3 = kV * kH, kB3 = kV;
constexpr int kParams = kW1 + kB1 + kW2 + kB2 + kW3 + kB3;  // 6,808

// Integer accumulators of one pass over a CSR matrix (all exact, so the result does not
// depend on the order of the atomic updates).
struct FeatAcc {
    unsigned long long sum_len, sum_len2, empty, band_sum, pairs, near_pairs, vertical;
    unsigned long long max_len, max_band;
};

__global__ void __launch_bounds__(256) features_pass_kernel(const int32_t *rowptr, const int32_t *colidx, int M,
                                                            int K, FeatAcc *acc) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    unsigned long long s_len = 0, s_len2 = 0, s_empty = 0, s_band = 0, s_pairs = 0, s_near = 0, s_vert = 0;
    unsigned long long m_len = 0, m_band = 0;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < M; row += warps) {
        const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
        const unsigned long long L = (unsigned long long)(p1 - p0);
        if (lane == 0) {
            s_len += L;
            s_len2 += L * L;
            s_empty += L == 0;
            s_pairs += L > 0 ? L - 1 : 0;
            m_len = L > m_len ? L : m_len;
        }
        const int64_t centre = (int64_t)row * K / M;
        const int64_t q0 = row + 1 < M ? rowptr[row + 1] : 0, q1 = row + 1 < M ? rowptr[row + 2] : 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int j = colidx[p];
            const int64_t d = j > centre ? j - centre : centre - j;
            s_band += (unsigned long long)d;
            m_band = (unsigned long long)d > m_band ? (unsigned long long)d : m_band;
            if (p + 1 < p1) {
                const int dj = colidx[p + 1] - j;
                s_near += (dj < 8 && dj > -8) ? 1 : 0;
            }
            // is column j stored in the next row (rows sorted by column)?
            int64_t lo = q0, hi = q1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (colidx[mid] < j) lo = mid + 1;
                else hi = mid;
            }
            s_vert += (lo < q1 && colidx[lo] == j) ? 1 : 0;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s_len += __shfl_xor_sync(FULL, s_len, off);
        s_len2 += __shfl_xor_sync(FULL, s_len2, off);
        s_empty += __shfl_xor_sync(FULL, s_empty, off);
        s_band += __shfl_xor_sync(FULL, s_band, off);
        s_pairs += __shfl_xor_sync(FULL, s_pairs, off);
        s_near += __shfl_xor_sync(FULL, s_near, off);
        s_vert += __shfl_xor_sync(FULL, s_vert, off);
        const unsigned long long a = __shfl_xor_sync(FULL, m_len, off), b = __shfl_xor_sync(FULL, m_band, off);
        m_len = a > m_len ? a : m_len;
        m_band = b > m_band ? b : m_band;
    }
    if (lane == 0) {
        atomicAdd(&acc->sum_len, s_len);
        atomicAdd(&acc->sum_len2, s_len2);
        atomicAdd(&acc->empty, s_empty);
        atomicAdd(&acc->band_sum, s_band);
        atomicAdd(&acc->pairs, s_pairs);
        atomicAdd(&acc->near_pairs, s_near);
        atomicAdd(&acc->vertical, s_vert);
        atomicMax(&acc->max_len, m_len);
        atomicMax(&acc->max_band, m_band);
    }
}

// The 16 features from the counters (FP64 on one thread, stored as FP32).
__global__ void features_finish_kernel(const FeatAcc *a, int M, int K, int N, int dtype, float *f) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double m = M, k = K, nnz = (double)a->sum_len;
    const double mean = M > 0 ? nnz / m : 0.0;
    const double var = M > 0 ? fmax((double)a->sum_len2 / m - mean * mean, 0.0) : 0.0;
    const double sd = sqrt(var);
    const double mx = (double)a->max_len;
    f[0] = (float)log2(fmax(m, 1.0));
    f[1] = (float)log2(fmax(k, 1.0));
    f[2] = (float)log2(1.0 + nnz);
    f[3] = (float)log2(fmax(nnz, 1.0) / (fmax(m, 1.0) * fmax(k, 1.0)));
    f[4] = (float)log2(1.0 + mean);
    f[5] = (float)log2(1.0 + sd);
    f[6] = (float)(mean > 0 ? sd / mean : 0.0);
    f[7] = (float)log2(1.0 + mx);
    f[8] = (float)(mean > 0 ? mx / mean : 0.0);
    f[9] = (float)(M > 0 ? (double)a->empty / m : 0.0);
    f[10] = (float)(nnz > 0 && K > 0 ? (double)a->band_sum / nnz / k : 0.0);
    f[11] = (float)(K > 0 ? (double)a->max_band / k : 0.0);
    f[12] = (float)(a->pairs > 0 ? (double)a->near_pairs / (double)a->pairs : 0.0);
    f[13] = (float)(nnz > 0 ? (double)a->vertical / nnz : 0.0);
    f[14] = (float)log2(fmax((double)N, 1.0));
    f[15] = (float)dtype;
}

// ---- MLP ------------------------------------------------------------------------------------
// Parameter layout (row-major, out x in): W1 [64 x 16], b1 [64], W2 [64 x 64], b2 [64],
// W3 [24 x 64], b3 [24].  Inputs are standardised with norm[0..15] (mean) and
// norm[16..31] (standard deviation).

struct Params {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__device__ __forceinline__ Params split(const float *w) {
    return Params{w, w + kW1, w + kW1 + kB1, w + kW1 + kB1 + kW2, w + kW1 + kB1 + kW2 + kB2,
                  w + kW1 + kB1 + kW2 + kB2 + kW3};
}

// Forward of one sample by one warp: x (16) -> h1 (64) -> h2 (64) -> y (24).  Each output
// is one lane's plain dot product in input order.
__device__ void forward_one(const Params &P, const float *x, float *h1, float *h2, float *y, int lane) {
    for (int o = lane; o < kH; o += 32) {
        float s = P.b1[o];
        for (int i = 0; i < kF; ++i) s = fmaf(P.W1[o * kF + i], x[i], s);
        h1[o] = fmaxf(s, 0.f);
    }
    __syncwarp();
    for (int o = lane; o < kH; o += 32) {
        float s = P.b2[o];
        for (int i = 0; i < kH; ++i) s = fmaf(P.W2[o * kH + i], h1[i], s);
        h2[o] = fmaxf(s, 0.f);
    }
    __syncwarp();
    for (int o = lane; o < kV; o += 32) {
        float s = P.b3[o];
        for (int i = 0; i < kH; ++i) s = fmaf(P.W3[o * kH + i], h2[i], s);
        y[o] = s;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) mlp_predict_kernel(const float *w, const float *norm, const float *feats, int n,
                                                          float *out, int32_t *choice) {
    __shared__ float buf[8][kF + kH + kH + kV];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int s = blockIdx.x * 8 + wi;
    if (s >= n) return;
    float *x = buf[wi], *h1 = x + kF, *h2 = h1 + kH, *y = h2 + kH;
    if (lane < kF) x[lane] = (feats[(int64_t)s * kF + lane] - norm[lane]) / norm[kF + lane];
    __syncwarp();
    const Params P = split(w);
    forward_one(P, x, h1, h2, y, lane);
    if (out && lane < kV) out[(int64_t)s * kV + lane] = y[lane];
    if (choice && lane == 0) {
        int best = 0;
        for (int v = 1; v < kV; ++v)
            if (y[v] < y[best]) best = v;
        choice[s] = best;
    }
}

// Mean and standard deviation (population, 1 if zero) of each feature over n samples.
__global__ void feature_norm_kernel(const float *feats, int n, float *norm) {
    const int f = threadIdx.x;
    if (f >= kF) return;
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
        const double v = feats[(int64_t)i * kF + f];
        s += v;
        s2 += v * v;
    }
    const double mean = n > 0 ? s / n : 0.0;
    const double var = n > 0 ? fmax(s2 / n - mean * mean, 0.0) : 0.0;
    norm[f] = (float)mean;
    norm[kF + f] = var > 0 ? (float)sqrt(var) : 1.0f;
}

// `steps` Adam steps on minibatches of `batch` samples taken in turn from order[]:
// loss = sum over samples and valid outputs (mask 1) of (y - target)^2 / (number of valid
// outputs in the batch).  One CTA; gradients are sums over the batch in sample order.
// adam holds m then v (kParams each); t0 is the number of steps already taken.
constexpr int kMaxBatch = 64;
__global__ void __launch_bounds__(256) mlp_train_kernel(float *w, float *adam, const float *norm, const float *feats,
                                                        const float *targets, const float *mask, const int32_t *order,
                                                        int norder, int steps, int batch, float lr, int t0) {
    extern __shared__ float sm[];
    float *X = sm;                     // batch x 16
    float *H1 = X + kMaxBatch * kF;    // batch x 64
    float *H2 = H1 + kMaxBatch * kH;   // batch x 64
    float *Y = H2 + kMaxBatch * kH;    // batch x 24, then dL/dy
    float *D2 = Y + kMaxBatch * kV;    // batch x 64: dL/dh2 (pre-activation)
    float *D1 = D2 + kMaxBatch * kH;   // batch x 64: dL/dh1 (pre-activation)
    float *G = D1 + kMaxBatch * kH;    // kParams gradients
    __shared__ float s_count;
    const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
    const Params P = split(w);
    const float b1c = 0.9f, b2c = 0.999f, eps = 1e-8f;
    for (int step = 0; step < steps; ++step) {
        const int base = (int)(((int64_t)step * batch) % norder);
        // inputs
        for (int e = tid; e < batch * kF; e += blockDim.x) {
            const int b = e / kF, f = e % kF;
            const int s = order[(base + b) % norder];
            X[e] = (feats[(int64_t)s * kF + f] - norm[f]) / norm[kF + f];
        }
        __syncthreads();
        // forward, one warp per sample
        for (int b = wi; b < batch; b += blockDim.x / 32)
            forward_one(P, X + b * kF, H1 + b * kH, H2 + b * kH, Y + b * kV, lane);
        __syncthreads();
        if (tid == 0) {
            float c = 0.f;
            for (int b = 0; b < batch; ++b) {
                const int s = order[(base + b) % norder];
                for (int v = 0; v < kV; ++v) c += mask[(int64_t)s * kV + v];
            }
            s_count = c > 0.f ? c : 1.f;
        }
        __syncthreads();
        // dL/dy
        for (int e = tid; e < batch * kV; e += blockDim.x) {
            const int b = e / kV, v = e % kV;
            const int s = order[(base + b) % norder];
            const float mk = mask[(int64_t)s * kV + v];
            Y[e] = mk * 2.f * (Y[e] - targets[(int64_t)s * kV + v]) / s_count;
        }
        __syncthreads();
        // dL/dh2 (through ReLU)
        for (int e = tid; e < batch * kH; e += blockDim.x) {
            const int b = e / kH, i = e % kH;
            float s = 0.f;
            for (int v = 0; v < kV; ++v) s = fmaf(P.W3[v * kH + i], Y[b * kV + v], s);
            D2[e] = H2[e] > 0.f ? s : 0.f;
        }
        __syncthreads();
        // dL/dh1 (through ReLU)
        for (int e = tid; e < batch * kH; e += blockDim.x) {
            const int b = e / kH, i = e % kH;
            float s = 0.f;
            for (int o = 0; o < kH; ++o) s = fmaf(P.W2[o * kH + i], D2[b * kH + o], s);
            D1[e] = H1[e] > 0.f ? s : 0.f;
        }
        __syncthreads();
        // parameter gradients: each is a sum over the batch in sample order
        for (int e = tid; e < kParams; e += blockDim.x) {
            float g = 0.f;
            if (e < kW1) {
                const int o = e / kF, i = e % kF;
                for (int b = 0; b < batch; ++b) g = fmaf(D1[b * kH + o], X[b * kF + i], g);
            } else if (e < kW1 + kB1) {
                const int o = e - kW1;
                for (int b = 0; b < batch; ++b) g += D1[b * kH + o];
            } else if (e < kW1 + kB1 + kW2) {
                const int q = e - kW1 - kB1, o = q / kH, i = q % kH;
                for (int b = 0; b < batch; ++b) g = fmaf(D2[b * kH + o], H1[b * kH + i], g);
            } else if (e < kW1 + kB1 + kW2 + kB2) {
                const int o = e - kW1 - kB1 - kW2;
                for (int b = 0; b < batch; ++b) g += D2[b * kH + o];
            } else if (e < kW1 + kB1 + kW2 + kB2 + kW3) {
                const int q = e - kW1 - kB1 - kW2 - kB2, v = q / kH, i = q % kH;
                for (int b = 0; b < batch; ++b) g = fmaf(Y[b * kV + v], H2[b * kH + i], g);
            } else {
                const int v = e - kW1 - kB1 - kW2 - kB2 - kW3;
                for (int b = 0; b < batch; ++b) g += Y[b * kV + v];
            }
            G[e] = g;
        }
        __syncthreads();
        // Adam
        const int t = t0 + step + 1;
        const float c1 = 1.f - powf(b1c, (float)t), c2 = 1.f - powf(b2c, (float)t);
        for (int e = tid; e < kParams; e += blockDim.x) {
            const float g = G[e];
            const float m = b1c * adam[e] + (1.f - b1c) * g;
            const float v = b2c * adam[kParams + e] + (1.f - b2c) * g * g;
            adam[e] = m;
            adam[kParams + e] = v;
            w[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
        __syncthreads();
    }
}

}  // namespace sel

// The 24 SpMM variants the selector chooses among (index -> options):
//   0..8   row-split, vecs {1,2,4} x unroll {2,4,8}
//   9..17  merge path, vecs {1,2,4} x unroll {2,4,8}
//   18..20 merge path with 1 CTA per SM, vecs {1,2}, and with 2 CTAs per SM, vecs 1; unroll 4
//   21     the SELL-C-sigma plan, C = 64, one sort window (gbsp_sell_plan_*; FP32 only),
//          variant GBSP_VARIANT_SELL_PLAN
//   22     row groups (several short rows per warp), default layout
//   23     the hyper-sparse plan (gbsp_hsp_plan_*; FP32 only), variant GBSP_VARIANT_HSP_PLAN
int variant_opts(int v, gbsp_opts *o) {
    static const int vecs[3] = {1, 2, 4}, unr[3] = {2, 4, 8};
    *o = gbsp_opts{};
    if (v >= 0 && v < 18) {
        o->variant = v < 9 ? GBSP_VARIANT_ROWSPLIT : GBSP_VARIANT_MERGE;
        o->vecs = vecs[(v % 9) / 3];
        o->unroll = unr[v % 3];
        return GBSP_OK;
    }
    if (v >= 18 && v < 21) {
        o->variant = GBSP_VARIANT_MERGE;
        o->ctas_per_sm = 1 + (v - 18) / 2;
        o->vecs = 1 + (v - 18) % 2;
        o->unroll = 4;
        return GBSP_OK;
    }
    if (v == 21) {
        o->variant = GBSP_VARIANT_SELL_PLAN;
        return GBSP_OK;
    }
    if (v == 22) {
        o->variant = GBSP_VARIANT_ROWGROUP;
        return GBSP_OK;
    }
    if (v == 23) {
        o->variant = GBSP_VARIANT_HSP_PLAN;
        return GBSP_OK;
    }
    return fail(GBSP_ERR_INVALID_ARG, "variant index %d outside 0..23", v);
}

}  // namespace gbsp

using namespace gbsp;
using namespace gbsp::sel;

GBSP_EXPORT int gbsp_variant_opts(int variant, gbsp_opts *out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "variant_opts: null output");
    int st = variant_opts(variant, out);
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_features(const gbsp_csr *A, int64_t N, int32_t dtype, float *feats, void *stream) {
    if (!A || !feats || A->rows < 0 || A->cols < 0 || A->rows > 2147483647LL || A->cols > 2147483647LL ||
        (A->rows > 0 && (!A->rowptr || (A->nnz != 0 && !A->colidx))) || N < 0)
        return fail(GBSP_ERR_INVALID_ARG, "features: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *acc = nullptr;
    int st = scratch_alloc(&acc, sizeof(FeatAcc), s);
    if (st) return st;
    cudaMemsetAsync(acc, 0, sizeof(FeatAcc), s);
    if (A->rows > 0) {
        int64_t blocks = (A->rows + 7) / 8;
        if (blocks > 32L * sm_count()) blocks = 32L * sm_count();
        features_pass_kernel<<<(unsigned)blocks, 256, 0, s>>>(A->rowptr, A->colidx, (int)A->rows, (int)A->cols,
                                                               static_cast<FeatAcc *>(acc));
        count_launches(1);
    }
    features_finish_kernel<<<1, 32, 0, s>>>(static_cast<FeatAcc *>(acc), (int)A->rows, (int)A->cols, (int)N, dtype,
                                            feats);
    count_launches(1);
    st = check_launch("features");
    scratch_free(acc, s);
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_feature_norm(const float *feats, int n, float *norm, void *stream) {
    if (!feats || !norm || n < 0) return fail(GBSP_ERR_INVALID_ARG, "feature_norm: bad arguments");
    feature_norm_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(feats, n, norm);
    count_launches(1);
    int st = check_launch("feature_norm");
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_mlp_predict(const float *weights, const float *norm, const float *feats, int n, float *out,
                                 int32_t *choice, void *stream) {
    if (!weights || !norm || !feats || n < 0) return fail(GBSP_ERR_INVALID_ARG, "mlp_predict: bad arguments");
    if (n == 0) return ok();
    mlp_predict_kernel<<<(n + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(weights, norm, feats, n, out, choice);
    count_launches(1);
    int st = check_launch("mlp_predict");
    return st ? st : ok();
}

GBSP_EXPORT int gbsp_mlp_train(float *weights, float *adam, const float *norm, const float *feats,
                               const float *targets, const float *mask, const int32_t *order, int norder, int steps,
                               int batch, float lr, int t0, void *stream) {
    if (!weights || !adam || !norm || !feats || !targets || !mask || !order || norder <= 0 || steps < 0 ||
        batch < 1 || batch > kMaxBatch)
        return fail(GBSP_ERR_INVALID_ARG, "mlp_train: bad arguments (batch 1..%d)", kMaxBatch);
    const size_t smem = sizeof(float) * ((size_t)kMaxBatch * (kF + 4 * kH + kV) + kParams);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return check_launch("mlp_train attribute");
        attr = true;
    }
    mlp_train_kernel<<<1, 256, smem, static_cast<cudaStream_t>(stream)>>>(weights, adam, norm, feats, targets, mask,
                                                                          order, norder, steps, batch, lr, t0);
    count_launches(1);
    int st = check_launch("mlp_train");
    return st ? st : ok();
}

namespace {

// Times one variant: an untimed call (which also says whether the variant applies), then
// reps calls between two events.  Returns false when the variant does not apply.
template <class F>
bool time_variant(F call, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms_out, int *st) {
    if (call() != GBSP_OK) return false;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) call();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
        *st = check_launch("autotune");
        return false;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / reps;
    return true;
}

}  // namespace

GBSP_EXPORT int gbsp_autotune(const gbsp_csr *A, const gbsp_dense *B, gbsp_dense *C, int reps, float *times_ms,
                              int32_t *best, void *stream) {
    if (!A || !B || !C || !times_ms || reps < 1) return fail(GBSP_ERR_INVALID_ARG, "autotune: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return check_launch("autotune events");
    int bi = -1;
    int st = GBSP_OK;
    for (int v = 0; v < kV && st == GBSP_OK; ++v) {
        gbsp_opts o;
        variant_opts(v, &o);
        times_ms[v] = INFINITY;
        float ms = 0.f;
        bool ran;
        if (o.variant == GBSP_VARIANT_HSP_PLAN) {
            // the plan is built outside the timed calls, as a caller builds it once per pattern
            gbsp_hsp_plan *plan = nullptr;
            if (A->dtype != GBSP_F32 || B->dtype != GBSP_F32 || A->nnz < 0 ||
                gbsp_hsp_plan_create(A, stream, &plan) != GBSP_OK)
                continue;
            ran = time_variant([&] { return gbsp_hsp_plan_execute(plan, B, C, stream); }, reps, s, e0, e1, &ms, &st);
            gbsp_hsp_plan_destroy(plan);
        } else if (o.variant == GBSP_VARIANT_SELL_PLAN) {
            gbsp_sell_plan *plan = nullptr;
            if (A->dtype != GBSP_F32 || B->dtype != GBSP_F32 || A->nnz < 0 ||
                gbsp_sell_plan_create(A, 64, 0, stream, &plan) != GBSP_OK)
                continue;
            ran = time_variant([&] { return gbsp_sell_plan_execute(plan, B, C, stream); }, reps, s, e0, e1, &ms, &st);
            gbsp_sell_plan_destroy(plan);
        } else {
            ran = time_variant([&] { return spmm_csr_ex(A, B, C, &o, stream); }, reps, s, e0, e1, &ms, &st);
        }
        if (!ran) continue;
        times_ms[v] = ms;
        if (bi < 0 || times_ms[v] < times_ms[bi]) bi = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (best) *best = bi;
    ok();  // a variant that did not apply left its message; the search itself succeeded
    return bi < 0 ? fail(GBSP_ERR_UNSUPPORTED, "autotune: no variant ran") : GBSP_OK;
}

// The SDDMM variants the selector chooses among: index 3 * split + (vecs index), split in
// {row split, merge path, entry split}, vecs {1, 2, 4}; indices 9..23 are unused.
GBSP_EXPORT int gbsp_sddmm_variant_opts(int variant, gbsp_opts *out) {
    if (!out) return fail(GBSP_ERR_INVALID_ARG, "sddmm_variant_opts: null output");
    if (variant < 0 || variant >= kSddmmVariants)
        return fail(GBSP_ERR_INVALID_ARG, "sddmm_variant_opts: index %d outside 0..%d", variant, kSddmmVariants - 1);
    static const int splits[3] = {GBSP_VARIANT_ROWSPLIT, GBSP_VARIANT_MERGE, GBSP_VARIANT_ENTRY};
    static const int vecs[3] = {1, 2, 4};
    *out = gbsp_opts{};
    out->variant = splits[variant / 3];
    out->vecs = vecs[variant % 3];
    return ok();
}

GBSP_EXPORT int gbsp_autotune_sddmm(const gbsp_csr *S, const gbsp_dense *X, const gbsp_dense *Y, float *out, int reps,
                                    float *times_ms, int32_t *best, void *stream) {
    if (!S || !X || !Y || !out || !times_ms || reps < 1)
        return fail(GBSP_ERR_INVALID_ARG, "autotune_sddmm: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return check_launch("autotune events");
    int bi = -1;
    int st = GBSP_OK;
    for (int v = 0; v < kV && st == GBSP_OK; ++v) {
        times_ms[v] = INFINITY;
        if (v >= kSddmmVariants) continue;
        gbsp_opts o;
        gbsp_sddmm_variant_opts(v, &o);
        float ms = 0.f;
        if (!time_variant([&] { return sddmm_csr_ex(S, X, Y, out, &o, stream); }, reps, s, e0, e1, &ms, &st))
            continue;
        times_ms[v] = ms;
        if (bi < 0 || times_ms[v] < times_ms[bi]) bi = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (best) *best = bi;
    ok();
    return bi < 0 ? fail(GBSP_ERR_UNSUPPORTED, "autotune_sddmm: no variant ran") : GBSP_OK;
}

// Batched FP64 GEMM launchers and the descriptor staging buffers of a context.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "gemm.cuh"

namespace tlr {

void *stage_push(tlr_ctx *ctx, const void *data, size_t bytes, cudaStream_t s) {
    StageRing &R = ctx->stage[stage_ring(ctx, s)];
    size_t need = (bytes + 255) & ~(size_t)255;
    if (need > R.cap) throw make_error(TLR_ERR_ARG, "descriptor batch too large (%zu bytes)", bytes);
    if (R.off + need > R.cap) {
        // every reader of this ring runs on `s`
        TLR_CUDA_TRY(cudaStreamSynchronize(s));
        R.off = 0;
    }
    char *h = R.h + R.off;
    char *d = R.d + R.off;
    std::memcpy(h, data, bytes);
    TLR_CUDA_TRY(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s));
    R.off += need;
    return d;
}

template <int BM, int BN, class Epi>
static void launch_shape(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                         double alpha, const Epi &epi, bool df) {
    if (probs.empty()) return;
    std::vector<int> off(probs.size() + 1, 0);
    for (size_t b = 0; b < probs.size(); ++b) {
        const GemmProb &p = probs[b];
        int tiles = (p.m > 0 && p.n > 0) ? (int)(ceil_div(p.m, BM) * ceil_div(p.n, BN)) : 0;
        off[b + 1] = off[b] + tiles;
    }
    int total = off.back();
    if (total == 0) return;
    auto *dp = (const GemmProb *)stage_push(ctx, probs.data(), probs.size() * sizeof(GemmProb), s);
    auto *dt = (const int *)stage_push(ctx, off.data(), off.size() * sizeof(int), s);
    int np = (int)probs.size();
    // the transposition pairs the library uses: NN, TN, NT (no TT)
    if (ta && tb) throw make_error(TLR_ERR_ARG, "GEMM with both operands transposed is not provided");
    if (df) {
        if (!ta && !tb) launch(k_gemm_df<BM, BN, false, false, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
        else if (!ta) launch(k_gemm_df<BM, BN, false, true, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
        else launch(k_gemm_df<BM, BN, true, false, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
    } else if (!ta && !tb) launch(k_gemm_f64<BM, BN, false, false, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
    else if (!ta) launch(k_gemm_f64<BM, BN, false, true, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
    else launch(k_gemm_f64<BM, BN, true, false, Epi>, total, kGemmThreads, 0, s, dp, dt, np, total, alpha, epi);
    TLR_CHECK_LAUNCH();
}

static void launch_gemv(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                        double alpha, const EpiLinear &epi) {
    if (probs.empty()) return;
    std::vector<int> off(probs.size() + 1, 0);
    for (size_t b = 0; b < probs.size(); ++b)
        off[b + 1] = off[b] + (probs[b].m > 0 ? (int)ceil_div(probs[b].m, kGemvRows) : 0);
    int total = off.back();
    if (total == 0) return;
    auto *dp = (const GemmProb *)stage_push(ctx, probs.data(), probs.size() * sizeof(GemmProb), s);
    auto *dt = (const int *)stage_push(ctx, off.data(), off.size() * sizeof(int), s);
    int np = (int)probs.size();
    if (ta && tb) launch(k_gemv<true, true>, total, kGemmThreads, 0, s, dp, dt, np, alpha, epi);
    else if (ta) launch(k_gemv<true, false>, total, kGemmThreads, 0, s, dp, dt, np, alpha, epi);
    else if (tb) launch(k_gemv<false, true>, total, kGemmThreads, 0, s, dp, dt, np, alpha, epi);
    else launch(k_gemv<false, false>, total, kGemmThreads, 0, s, dp, dt, np, alpha, epi);
    TLR_CHECK_LAUNCH();
}

// Split a batch by output shape: problems with at most 32 rows and/or 32
// columns go to the thin tile shapes, whose padding stays small; FP64
// matrix-vector products (n = 1) go to the GEMV kernel.
template <class Epi>
static void launch_gemm(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                        double alpha, const Epi &epi, bool df) {
    std::vector<GemmProb> cls[4];  // 64x64, 64x32, 32x64, 32x32
    if constexpr (std::is_same<Epi, EpiLinear>::value) {
        if (!df) {
            std::vector<GemmProb> vec, rest;
            for (const GemmProb &p : probs) (p.n == 1 ? vec : rest).push_back(p);
            launch_gemv(ctx, s, ta, tb, vec, alpha, epi);
            for (const GemmProb &p : rest) cls[(p.m <= 32 ? 2 : 0) + (p.n <= 32 ? 1 : 0)].push_back(p);
            launch_shape<64, 64>(ctx, s, ta, tb, cls[0], alpha, epi, df);
            launch_shape<64, 32>(ctx, s, ta, tb, cls[1], alpha, epi, df);
            launch_shape<32, 64>(ctx, s, ta, tb, cls[2], alpha, epi, df);
            launch_shape<32, 32>(ctx, s, ta, tb, cls[3], alpha, epi, df);
            return;
        }
    }
    for (const GemmProb &p : probs) cls[(p.m <= 32 ? 2 : 0) + (p.n <= 32 ? 1 : 0)].push_back(p);
    launch_shape<64, 64>(ctx, s, ta, tb, cls[0], alpha, epi, df);
    launch_shape<64, 32>(ctx, s, ta, tb, cls[1], alpha, epi, df);
    launch_shape<32, 64>(ctx, s, ta, tb, cls[2], alpha, epi, df);
    launch_shape<32, 32>(ctx, s, ta, tb, cls[3], alpha, epi, df);
}

__global__ void k_split_f2(const double *__restrict__ src, int ld, int m, int64_t count,
                           float2 *__restrict__ dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    int64_t i = e % m, j = e / m;
    double v = src[j * ld + i];
    float h = __double2float_rn(v);
    dst[j * ld + i] = make_float2(h, __double2float_rn(v - (double)h));
}

void split_f2(cudaStream_t s, const double *src, int ld, int m, int n, float2 *dst) {
    int64_t count = (int64_t)m * n;
    if (count <= 0) return;
    launch(k_split_f2, (unsigned)ceil_div(count, 256), 256, 0, s, src, ld, m, count, dst);
    TLR_CHECK_LAUNCH();
}

// blockIdx.y: descriptor; blockIdx.x strides over its columns, threads over rows.
__global__ void k_split_f2_batched(const SplitDesc *__restrict__ descs) {
    const SplitDesc D = descs[blockIdx.y];
    for (int j = blockIdx.x; j < D.n; j += gridDim.x) {
        const double *src = D.src + (int64_t)j * D.ld;
        float2 *dst = D.dst + (int64_t)j * D.ld;
        for (int i = threadIdx.x; i < D.m; i += blockDim.x) {
            const double v = src[i];
            const float h = __double2float_rn(v);
            dst[i] = make_float2(h, __double2float_rn(v - (double)h));
        }
    }
}

void split_f2_batched(tlr_ctx *ctx, cudaStream_t s, const std::vector<SplitDesc> &descs) {
    if (descs.empty()) return;
    int most = 0;
    for (const SplitDesc &d : descs) most = std::max(most, (d.m > 0) ? d.n : 0);
    if (most == 0) return;
    auto *dd = (const SplitDesc *)stage_push(ctx, descs.data(), descs.size() * sizeof(SplitDesc), s);
    dim3 grid((unsigned)std::min(most, 1024), (unsigned)descs.size());
    launch(k_split_f2_batched, grid, 256, 0, s, dd);
    TLR_CHECK_LAUNCH();
}

void gemm_batched_small(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                        double alpha, double beta) {
    launch_shape<32, 32>(ctx, s, ta, tb, probs, alpha, EpiLinear{beta}, false);
}

void gemm_batched(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                  double alpha, double beta, bool df) {
    launch_gemm(ctx, s, ta, tb, probs, alpha, EpiLinear{beta}, df);
}

// The panel update is one large product: 64 x 64 tiles.  A capped grid
// reserves more than half of an SM's shared memory per CTA (unused), so that
// each of its CTAs holds an SM of its own; ctas_per_sm = k reserves more than
// 1/(k+1) of it, so that at most k CTAs of this product share an SM and the
// rest of every SM stays open to the critical-path kernels on the
// high-priority streams.
template <class Epi>
static void launch_matern(tlr_ctx *ctx, cudaStream_t s, const std::vector<GemmProb> &big, double alpha,
                          const Epi &e, bool df, int max_ctas, int ctas_per_sm) {
    if (big.empty()) return;
    std::vector<int> off(big.size() + 1, 0);
    for (size_t b = 0; b < big.size(); ++b)
        off[b + 1] = off[b] + ((big[b].m > 0 && big[b].n > 0) ? (int)(ceil_div(big[b].m, 64) * ceil_div(big[b].n, 64)) : 0);
    int total = off.back();
    if (total == 0) return;
    auto *dp = (const GemmProb *)stage_push(ctx, big.data(), big.size() * sizeof(GemmProb), s);
    auto *dt = (const int *)stage_push(ctx, off.data(), off.size() * sizeof(int), s);
    int np = (int)big.size();
    const int grid = max_ctas > 0 ? std::min(total, max_ctas) : total;
    size_t smem = 0;
    const int per = max_ctas > 0 ? 1 : ctas_per_sm;
    if (per > 0) {
        static std::mutex mu;
        static size_t set_to = 0;
        int dev = 0, per_sm = 0;
        TLR_CUDA_TRY(cudaGetDevice(&dev));
        TLR_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        smem = (size_t)per_sm / (per + 1) + 1024;
        std::lock_guard<std::mutex> lock(mu);
        if (smem > set_to) {
            for (const void *k : {(const void *)k_gemm_df<64, 64, false, true, EpiMatern>,
                                  (const void *)k_gemm_f64<64, 64, false, true, EpiMatern>,
                                  (const void *)k_gemm_df<64, 64, false, true, EpiMaternMulti>,
                                  (const void *)k_gemm_f64<64, 64, false, true, EpiMaternMulti>})
                TLR_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            set_to = smem;
        }
    }
    if (df) launch(k_gemm_df<64, 64, false, true, Epi>, grid, kGemmThreads, smem, s, dp, dt, np, total, alpha, e);
    else launch(k_gemm_f64<64, 64, false, true, Epi>, grid, kGemmThreads, smem, s, dp, dt, np, total, alpha, e);
    TLR_CHECK_LAUNCH();
}

void gemm_batched_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs,
                         double alpha, const double *xy, int64_t n, const MaternParams &P, bool df, int max_ctas,
                         int ctas_per_sm) {
    if (!tb) throw make_error(TLR_ERR_ARG, "the Matern panel product takes B transposed");
    EpiMatern e;
    e.xy = xy;
    e.n = n;
    e.P = P;
    launch_matern(ctx, s, probs, alpha, e, df, max_ctas, ctas_per_sm);
}

void gemm_batched_matern_multi(tlr_ctx *ctx, cudaStream_t s, const std::vector<GemmProb> &probs, double alpha,
                               const std::vector<MaternItem> &items, bool df, int ctas_per_sm) {
    if (probs.empty() || items.empty()) return;
    EpiMaternMulti e;
    e.items = (const MaternItem *)stage_push(ctx, items.data(), items.size() * sizeof(MaternItem), s);
    launch_matern(ctx, s, probs, alpha, e, df, 0, ctas_per_sm);
}

}  // namespace tlr

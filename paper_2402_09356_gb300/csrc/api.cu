// C ABI of the TLR library (include/tlr.h).  Every entry point validates its
// arguments, runs its kernels on the caller's stream and turns any internal
// error into a status code plus a message in the context.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "common.cuh"
#include "compress.cuh"
#include "matern.cuh"
#include "tcgemm.cuh"
#include "tlr_internal.cuh"

namespace tlr {

std::atomic<long long> g_launch_count{0};

void status_reset(tlr_ctx *ctx, cudaStream_t s) {
    TLR_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), s));
}

int status_fetch(tlr_ctx *ctx, cudaStream_t s, long long *info) {
    TLR_CUDA_TRY(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) *info = ctx->h_status->info;
    return ctx->h_status->code;
}

void profile_events(tlr_ctx *ctx, int count) {
    while ((int)ctx->prof_events.size() < count) {
        cudaEvent_t e;
        TLR_CUDA_TRY(cudaEventCreate(&e));
        ctx->prof_events.push_back(e);
    }
}

static int fail(tlr_ctx *ctx, const Error &e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
}

template <class F>
static int guarded(tlr_ctx *ctx, F &&f) {
    if (!ctx) return TLR_ERR_ARG;
    try {
        TLR_CUDA_TRY(cudaSetDevice(ctx->device));
        ctx->err.clear();
        f();
        return TLR_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    } catch (const std::exception &e) {
        return fail(ctx, Error{TLR_ERR_CUDA, e.what()});
    }
}

static void check_arg(bool ok, const char *what) {
    if (!ok) throw make_error(TLR_ERR_ARG, "invalid argument: %s", what);
}

static MaternParams params_of(tlr_theta th) {
    MaternParams P;
    if (!make_matern_params(th.sigma2, th.beta, th.nu, &P))
        throw make_error(TLR_ERR_ARG, "theta must be positive and finite (sigma2=%g beta=%g nu=%g)",
                         th.sigma2, th.beta, th.nu);
    return P;
}

bool mle_bounds_ok(tlr_theta lo, tlr_theta hi) {
    return lo.sigma2 > 0 && lo.beta > 0 && lo.nu > 0 && hi.sigma2 >= lo.sigma2 && hi.beta >= lo.beta &&
           hi.nu >= lo.nu && std::isfinite(hi.sigma2) && std::isfinite(hi.beta) && std::isfinite(hi.nu);
}

void mle_nelder_mead(const std::function<double(tlr_theta)> &negll, tlr_theta theta0, tlr_theta lo,
                     tlr_theta hi, double tol, int max_iter, tlr_theta *theta_hat, double *ll_hat, int *iters) {
    const double llo[3] = {std::log(lo.sigma2), std::log(lo.beta), std::log(lo.nu)};
    const double lhi[3] = {std::log(hi.sigma2), std::log(hi.beta), std::log(hi.nu)};
    int evals = 0;
    auto clampv = [&](double *v) {
        for (int d = 0; d < 3; ++d) v[d] = std::min(lhi[d], std::max(llo[d], v[d]));
    };
    // the search runs in log(theta)
    auto f = [&](const double *v) -> double {
        ++evals;
        return negll(tlr_theta{std::exp(v[0]), std::exp(v[1]), std::exp(v[2])});
    };
    double x[4][3], fx[4];
    double v0[3] = {std::log(theta0.sigma2), std::log(theta0.beta), std::log(theta0.nu)};
    clampv(v0);
    for (int p = 0; p < 4; ++p) {
        for (int d = 0; d < 3; ++d) x[p][d] = v0[d];
        if (p > 0) x[p][p - 1] += 0.1;
        clampv(x[p]);
        fx[p] = f(x[p]);
    }
    // Nelder-Mead (reflection 1, expansion 2, contraction 1/2, shrink 1/2)
    while (evals < max_iter) {
        int idx[4] = {0, 1, 2, 3};
        std::sort(idx, idx + 4, [&](int a, int b) { return fx[a] < fx[b]; });
        double xs[4][3], fs[4];
        for (int p = 0; p < 4; ++p) {
            fs[p] = fx[idx[p]];
            for (int d = 0; d < 3; ++d) xs[p][d] = x[idx[p]][d];
        }
        std::memcpy(x, xs, sizeof x);
        std::memcpy(fx, fs, sizeof fx);
        if (std::isfinite(fx[3]) && std::fabs(fx[3] - fx[0]) <= tol * (1.0 + std::fabs(fx[0]))) break;
        double diam = 0.0;  // simplex size in log(theta)
        for (int p = 1; p < 4; ++p)
            for (int d = 0; d < 3; ++d) diam = std::max(diam, std::fabs(x[p][d] - x[0][d]));
        if (diam < 1e-8) break;
        double c[3] = {0, 0, 0};
        for (int p = 0; p < 3; ++p)
            for (int d = 0; d < 3; ++d) c[d] += x[p][d] / 3.0;
        double xr[3], xe[3], xc[3];
        for (int d = 0; d < 3; ++d) xr[d] = c[d] + (c[d] - x[3][d]);
        clampv(xr);
        double fr = f(xr);
        if (fr < fx[0]) {
            for (int d = 0; d < 3; ++d) xe[d] = c[d] + 2.0 * (c[d] - x[3][d]);
            clampv(xe);
            double fe = f(xe);
            if (fe < fr) { std::memcpy(x[3], xe, sizeof xe); fx[3] = fe; }
            else { std::memcpy(x[3], xr, sizeof xr); fx[3] = fr; }
        } else if (fr < fx[2]) {
            std::memcpy(x[3], xr, sizeof xr);
            fx[3] = fr;
        } else {
            bool outside = fr < fx[3];
            for (int d = 0; d < 3; ++d)
                xc[d] = outside ? c[d] + 0.5 * (xr[d] - c[d]) : c[d] + 0.5 * (x[3][d] - c[d]);
            clampv(xc);
            double fc = f(xc);
            if (fc < (outside ? fr : fx[3])) {
                std::memcpy(x[3], xc, sizeof xc);
                fx[3] = fc;
            } else {
                for (int p = 1; p < 4; ++p) {
                    for (int d = 0; d < 3; ++d) x[p][d] = x[0][d] + 0.5 * (x[p][d] - x[0][d]);
                    fx[p] = f(x[p]);
                }
            }
        }
    }
    int best = 0;
    for (int p = 1; p < 4; ++p)
        if (fx[p] < fx[best]) best = p;
    if (!std::isfinite(fx[best])) throw make_error(TLR_ERR_NOT_SPD, "no feasible likelihood evaluation");
    *theta_hat = tlr_theta{std::exp(x[best][0]), std::exp(x[best][1]), std::exp(x[best][2])};
    *ll_hat = -fx[best];
    *iters = evals;
}

}  // namespace tlr

using namespace tlr;

extern "C" {

const char *tlr_version(void) { return "tlr-gb300 0.1 sm_103a"; }

int64_t tlr_launch_count(void) { return g_launch_count.load(); }

int tlr_ctx_create(int device, tlr_ctx **out) {
    if (!out) return TLR_ERR_ARG;
    *out = nullptr;
    auto *ctx = new tlr_ctx();
    ctx->device = device;
    int rc = guarded(ctx, [&] {
        int count = 0;
        TLR_CUDA_TRY(cudaGetDeviceCount(&count));
        if (device < 0 || device >= count) throw make_error(TLR_ERR_ARG, "no CUDA device %d", device);
        TLR_CUDA_TRY(cudaSetDevice(device));
        TLR_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
        // the context's word, then one per factorisation of a group call
        TLR_CUDA_TRY(cudaMalloc(&ctx->d_status, (1 + kMaxGroup) * sizeof(DevStatus)));
        TLR_CUDA_TRY(cudaMemset(ctx->d_status, 0, (1 + kMaxGroup) * sizeof(DevStatus)));
        TLR_CUDA_TRY(cudaHostAlloc(&ctx->h_status, (1 + kMaxGroup) * sizeof(DevStatus), cudaHostAllocDefault));
        // the critical-path streams (diagonal POTRF, compression classes) get the
        // highest priority, so that the look-ahead panel GEMM fills in behind them
        int prio_lo = 0, prio_hi = 0;
        TLR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        TLR_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio_hi));
        TLR_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->la, cudaStreamNonBlocking, prio_lo));
        TLR_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->hp, cudaStreamNonBlocking, prio_hi));
        TLR_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->sv, cudaStreamNonBlocking, prio_hi));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_sv_fork, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_sv_done, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_hp_fork, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_hp_join, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_la_fork, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_la_join, cudaEventDisableTiming));
        for (cudaStream_t &c : ctx->cls_stream)
            TLR_CUDA_TRY(cudaStreamCreateWithPriority(&c, cudaStreamNonBlocking, prio_hi));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->cls_fork, cudaEventDisableTiming));
        for (cudaEvent_t &e : ctx->cls_join) TLR_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreate(&ctx->ev_a));
        TLR_CUDA_TRY(cudaEventCreate(&ctx->ev_b));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        TLR_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
        for (StageRing &R : ctx->stage) {
            R.cap = (size_t)16 << 20;
            TLR_CUDA_TRY(cudaHostAlloc(&R.h, R.cap, cudaHostAllocDefault));
            TLR_CUDA_TRY(cudaMalloc(&R.d, R.cap));
        }
        TLR_CUDA_TRY(cudaMalloc(&ctx->d_mtab, 2 * (size_t)kTabIntervals * kTabCoef * sizeof(double)));
        // workspaces come from the device's default stream-ordered pool; keep
        // what is freed cached there instead of returning it to the driver at
        // every synchronisation (a factorisation syncs once per tile column,
        // and re-mapping its per-column workspaces then costs milliseconds)
        cudaMemPool_t mp = nullptr;
        TLR_CUDA_TRY(cudaDeviceGetDefaultMemPool(&mp, device));
        uint64_t keep = UINT64_MAX;
        TLR_CUDA_TRY(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep));
    });
    if (rc != TLR_OK) {
        tlr_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return TLR_OK;
}

void tlr_ctx_destroy(tlr_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->la) cudaStreamDestroy(ctx->la);
    if (ctx->hp) cudaStreamDestroy(ctx->hp);
    if (ctx->sv) cudaStreamDestroy(ctx->sv);
    for (cudaEvent_t e : {ctx->ev_la_fork, ctx->ev_la_join, ctx->ev_hp_fork, ctx->ev_hp_join, ctx->ev_sv_fork,
                          ctx->ev_sv_done})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t c : ctx->cls_stream)
        if (c) cudaStreamDestroy(c);
    if (ctx->cls_fork) cudaEventDestroy(ctx->cls_fork);
    for (cudaEvent_t e : ctx->cls_join)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {ctx->ev_a, ctx->ev_b, ctx->ev_fork, ctx->ev_join})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->cls_time_events) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->comp_events) cudaEventDestroy(e);
    for (StageRing &R : ctx->stage) {
        if (R.h) cudaFreeHost(R.h);
        if (R.d) cudaFree(R.d);
    }
    if (ctx->d_omega) cudaFree(ctx->d_omega);
    if (ctx->d_omega2) cudaFree(ctx->d_omega2);
    if (ctx->d_potrf_scratch) cudaFree(ctx->d_potrf_scratch);
    if (ctx->d_mtab) cudaFree(ctx->d_mtab);
    delete ctx;
}

const char *tlr_last_error(const tlr_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tlr_ctx_set_buckets(tlr_ctx *ctx, const tlr_buckets *b) {
    return guarded(ctx, [&] {
        const tlr_buckets v = b ? *b : default_buckets();
        check_arg(buckets_ok(v), "bucket sizes must be 1, 2, 4, 8 or 16 and edges positive, nondecreasing");
        ctx->buckets = v;
    });
}

int tlr_ctx_get_buckets(const tlr_ctx *ctx, tlr_buckets *out) {
    if (!ctx || !out) return TLR_ERR_ARG;
    *out = ctx->buckets;
    return TLR_OK;
}

int tlr_order(tlr_ctx *ctx, const double *xy, int64_t n, int method, uint64_t seed, uint32_t flags,
              int64_t *perm, uint32_t *codes, double *xy_out, void *stream) {
    return guarded(ctx, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        check_arg(n >= 0 && n < ((int64_t)1 << 31), "n");
        check_arg(method >= TLR_ORDER_IDENTITY && method <= TLR_ORDER_MAXMIN, "method");
        check_arg((flags & ~TLR_ORDER_QUANTIZE) == 0, "flags");
        check_arg(n == 0 || (xy && perm), "xy/perm");
        if (n == 0) return;
        switch (method) {
        case TLR_ORDER_IDENTITY: order_identity(n, perm, s); break;
        case TLR_ORDER_RANDOM:
        case TLR_ORDER_MORTON:
        case TLR_ORDER_HILBERT: order_sfc(xy, n, method, seed, perm, codes, s); break;
        case TLR_ORDER_KDTREE: order_kdtree(xy, n, perm, s); break;
        case TLR_ORDER_MAXMIN: order_maxmin(xy, n, perm, s, ctx->num_sms); break;
        }
        if (xy_out) permute_xy(xy, perm, n, (flags & TLR_ORDER_QUANTIZE) ? 1 : 0, xy_out, s);
    });
}

int tlr_gather(tlr_ctx *ctx, const int64_t *perm, const double *src, int64_t n, double *dst, void *stream) {
    return guarded(ctx, [&] {
        check_arg(n >= 0 && (n == 0 || (perm && src && dst)), "gather");
        gather(perm, src, n, dst, (cudaStream_t)stream);
    });
}

int64_t tlr_tiles_size(int64_t n, int nb) {
    if (n <= 0 || nb <= 0) return 0;
    int64_t nt = (n + nb - 1) / nb;
    return nt * (nt + 1) / 2 * (int64_t)nb * nb;
}

int tlr_generate(tlr_ctx *ctx, const double *xy, int64_t n, int nb, tlr_theta theta, double *tiles,
                 void *stream) {
    return guarded(ctx, [&] {
        check_arg(n > 0 && xy && tiles, "n/xy/tiles");
        check_arg(nb >= 16 && nb <= kMaxTile, "nb");
        MaternParams P = params_of(theta);
        build_matern_table(&P, ctx->d_mtab, (cudaStream_t)stream);
        generate_tiles(xy, n, nb, P, tiles, (cudaStream_t)stream);
    });
}

int tlr_gemm_tc(tlr_ctx *ctx, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                int slices, void *stream) {
    return guarded(ctx, [&] {
        check_arg(m >= 0 && n >= 0 && k >= 0 && m < (1 << 30) && n < (1 << 30) && k < (1 << 30), "m/n/k");
        check_arg(!(trans_a && trans_b), "both operands transposed");
        check_arg(slices == 1 || slices == kTcSlicesDefault, "slices");
        if (m == 0 || n == 0) return;
        check_arg(C && ldc >= m && ldc < (1LL << 31), "C/ldc");
        if (k > 0) {
            check_arg(A && B, "A/B");
            check_arg(lda >= (trans_a ? k : m) && lda < (1LL << 31), "lda");
            check_arg(ldb >= (trans_b ? n : k) && ldb < (1LL << 31), "ldb");
        }
        status_reset(ctx, (cudaStream_t)stream);
        gemm_tc_single(ctx, (cudaStream_t)stream, trans_a != 0, trans_b != 0, (int)m, (int)n, (int)k, alpha, A,
                       (int)lda, B, (int)ldb, beta, C, (int)ldc, slices);
        long long info = -1;
        const int sc = status_fetch(ctx, (cudaStream_t)stream, &info);  // syncs the stream
        if (sc) throw make_error(sc, "tensor-core product: device status %d", sc);
    });
}

int tlr_matern(tlr_ctx *ctx, const double *d, int64_t m, tlr_theta theta, double *out, void *stream) {
    return guarded(ctx, [&] {
        check_arg(m >= 0 && (m == 0 || (d && out)), "d/out");
        MaternParams P = params_of(theta);
        matern_vec(d, m, P, out, (cudaStream_t)stream);
    });
}

// D, U, V and the rank map of a new matrix; `hint` (empty: uniform slots)
// sets a compact layout and the starting rank map.
static void mat_create_impl(tlr_ctx *ctx, int64_t n, int nb, int maxrank, const std::vector<int32_t> &hint,
                            tlr_mat **out) {
    check_arg(out != nullptr, "out");
    *out = nullptr;
    check_arg(n > 0 && nb >= 16 && nb <= kMaxTile, "n/nb");
    if (maxrank <= 0) maxrank = nb / 2;
    check_arg(maxrank <= nb, "maxrank");
    auto *M = new tlr_mat();
    M->device = ctx->device;
    M->n = n;
    M->nb = nb;
    M->nt = (int)((n + nb - 1) / nb);
    M->maxrank = maxrank;
    const int64_t cols = plan_slots(M, hint);
    size_t dbytes = (size_t)M->nt * nb * nb * sizeof(double);
    size_t uvbytes = (size_t)cols * nb * sizeof(double);
    size_t rbytes = (size_t)M->nt * M->nt * sizeof(int32_t);
    cudaError_t e1 = cudaMalloc(&M->D, dbytes);
    cudaError_t e2 = cudaMalloc(&M->U, uvbytes);
    cudaError_t e3 = cudaMalloc(&M->V, uvbytes);
    cudaError_t e4 = cudaMalloc(&M->ranks, rbytes);
    if (e1 || e2 || e3 || e4) {
        tlr_mat_destroy(M);
        cudaGetLastError();
        throw make_error(TLR_ERR_OOM, "cannot allocate TLR matrix (%zu + 2 x %zu bytes)", dbytes, uvbytes);
    }
    M->bytes = dbytes + 2 * uvbytes + rbytes;
    // padding rows of U / V must read as zero
    TLR_CUDA_TRY(cudaMemset(M->D, 0, dbytes));
    TLR_CUDA_TRY(cudaMemset(M->U, 0, uvbytes));
    TLR_CUDA_TRY(cudaMemset(M->V, 0, uvbytes));
    TLR_CUDA_TRY(cudaMemset(M->ranks, 0, rbytes));
    M->h_ranks = hint;
    *out = M;
}

int tlr_mat_create(tlr_ctx *ctx, int64_t n, int nb, int maxrank, tlr_mat **out) {
    return guarded(ctx, [&] { mat_create_impl(ctx, n, nb, maxrank, {}, out); });
}

int tlr_mat_create_compact(tlr_ctx *ctx, int64_t n, int nb, int maxrank, const int32_t *rank_map, tlr_mat **out) {
    return guarded(ctx, [&] {
        check_arg(rank_map != nullptr && n > 0 && nb > 0, "rank_map");
        const int64_t nt = (n + nb - 1) / nb;
        std::vector<int32_t> hint(rank_map, rank_map + nt * nt);
        for (int64_t t = 0; t < nt; ++t) hint[(size_t)(t * nt + t)] = (int32_t)std::min<int64_t>(nb, n - t * nb);
        mat_create_impl(ctx, n, nb, maxrank, hint, out);
    });
}

int64_t tlr_mat_bytes(const tlr_mat *M) { return M ? (int64_t)M->bytes : 0; }

int64_t tlr_mat_plan_bytes(int64_t n, int nb, int maxrank, const int32_t *rank_map) {
    if (n <= 0 || nb < 16 || nb > kMaxTile || maxrank > nb) return -1;
    tlr_mat M;
    M.n = n;
    M.nb = nb;
    M.nt = (int)((n + nb - 1) / nb);
    M.maxrank = maxrank > 0 ? maxrank : nb / 2;
    std::vector<int32_t> hint;
    if (rank_map) hint.assign(rank_map, rank_map + (size_t)M.nt * M.nt);
    const int64_t cols = plan_slots(&M, hint);
    return ((int64_t)M.nt * nb * nb + 2 * cols * nb) * (int64_t)sizeof(double) + (int64_t)M.nt * M.nt * 4;
}

void tlr_mat_destroy(tlr_mat *M) {
    if (!M) return;
    cudaSetDevice(M->device);
    cudaDeviceSynchronize();
    if (M->D) cudaFree(M->D);
    if (M->U) cudaFree(M->U);
    if (M->V) cudaFree(M->V);
    if (M->ranks) cudaFree(M->ranks);
    delete M;
}

int tlr_mat_layout(const tlr_mat *M, int64_t *n, int *nb, int *nt, int *maxrank, double **D, double **U,
                   double **V, int32_t **ranks) {
    if (!M) return TLR_ERR_ARG;
    if (n) *n = M->n;
    if (nb) *nb = M->nb;
    if (nt) *nt = M->nt;
    if (maxrank) *maxrank = M->maxrank;
    if (D) *D = M->D;
    if (U) *U = M->U;
    if (V) *V = M->V;
    if (ranks) *ranks = M->ranks;
    return TLR_OK;
}

int tlr_mat_tile(tlr_ctx *ctx, const tlr_mat *M, int i, int j, double *a, double *b, int32_t *rank,
                 void *stream) {
    return guarded(ctx, [&] {
        check_arg(M && a && rank, "mat/a/rank");
        check_arg(i >= 0 && j >= 0 && i < M->nt && j <= i, "tile index");
        cudaStream_t s = (cudaStream_t)stream;
        size_t nb = M->nb;
        if (i == j) {
            TLR_CUDA_TRY(cudaMemcpyAsync(a, M->D + (int64_t)i * nb * nb, nb * nb * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            *rank = tile_rows(M->n, M->nb, i);
            return;
        }
        check_arg(b != nullptr, "b");
        int r = M->h_ranks.size() == (size_t)M->nt * M->nt ? M->h_ranks[(size_t)i * M->nt + j] : 0;
        size_t off = (size_t)slot_col(M, i, j) * nb;
        if (r > 0) {
            TLR_CUDA_TRY(cudaMemcpyAsync(a, M->U + off, nb * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
            TLR_CUDA_TRY(cudaMemcpyAsync(b, M->V + off, nb * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        *rank = r;
    });
}

int tlr_mat_ranks(tlr_ctx *ctx, const tlr_mat *M, int32_t *host_ranks) {
    return guarded(ctx, [&] {
        check_arg(M && host_ranks, "mat/host_ranks");
        TLR_CUDA_TRY(cudaMemcpy(host_ranks, M->ranks, (size_t)M->nt * M->nt * sizeof(int32_t),
                                cudaMemcpyDeviceToHost));
    });
}

int tlr_compress(tlr_ctx *ctx, const double *tiles, int64_t n, int nb, double eps_abs, tlr_mat *A,
                 int64_t *info, void *stream) {
    long long inf = -1;
    int rc = guarded(ctx, [&] {
        check_arg(tiles && A, "tiles/A");
        check_arg(A->n == n && A->nb == nb, "A does not match n/nb");
        check_arg(eps_abs >= 0 && std::isfinite(eps_abs), "eps_abs");
        compress_packed(ctx, (cudaStream_t)stream, tiles, A, eps_abs, &inf);
    });
    if (info) *info = inf;
    return rc;
}

int tlr_potrf(tlr_ctx *ctx, tlr_mat *A, double eps_abs, int64_t *info, void *stream) {
    long long inf = -1;
    int rc = guarded(ctx, [&] {
        check_arg(A != nullptr, "A");
        check_arg(eps_abs >= 0 && std::isfinite(eps_abs), "eps_abs");
        cudaStream_t s = (cudaStream_t)stream;
        status_reset(ctx, s);
        FactorStats st;
        factor(ctx, s, A, FactorMode::Tlr, nullptr, nullptr, eps_abs, &st, &inf);
    });
    if (info) *info = inf;
    return rc;
}

int tlr_solve(tlr_ctx *ctx, const tlr_mat *L, const double *z, double *y, double *logdet, double *quad,
              void *stream) {
    return guarded(ctx, [&] {
        check_arg(L && z && y, "L/z/y");
        cudaStream_t s = (cudaStream_t)stream;
        check_arg(L->h_ranks.size() == (size_t)L->nt * L->nt, "L holds no factor");
        DevBuf acc(2 * sizeof(double), s);
        TLR_CUDA_TRY(cudaMemsetAsync(acc.as<double>(), 0, 2 * sizeof(double), s));
        status_reset(ctx, s);
        forward_solve(ctx, s, L, z, y, acc.as<double>());
        double h[2];
        TLR_CUDA_TRY(cudaMemcpyAsync(h, acc.as<double>(), sizeof h, cudaMemcpyDeviceToHost, s));
        TLR_CUDA_TRY(cudaStreamSynchronize(s));
        if (logdet) *logdet = 2.0 * h[0];
        if (quad) *quad = h[1];
    });
}

int tlr_lmul(tlr_ctx *ctx, const tlr_mat *L, const double *w, double *z, void *stream) {
    return guarded(ctx, [&] {
        check_arg(L && w && z && w != z, "L/w/z");
        check_arg(L->h_ranks.size() == (size_t)L->nt * L->nt, "L holds no factor");
        lmul(ctx, (cudaStream_t)stream, L, w, z);
    });
}

// Eq. 1.2 and the factor's rank statistics from acc = (sum log L_ii, |L^-1 z|^2,
// max 1 / L_ii^2) of a finished factorisation.
static void fill_result(tlr_result *out, int64_t n, const tlr_mat *L, const double *h, const FactorStats &st) {
    out->logdet = 2.0 * h[0];
    out->quad = h[1];
    out->min_pivot2 = h[2] > 0.0 ? 1.0 / h[2] : INFINITY;
    out->loglik = -0.5 * (double)n * std::log(2.0 * M_PI) - 0.5 * out->logdet - 0.5 * out->quad;
    if (!std::isfinite(out->loglik)) throw make_error(TLR_ERR_NAN, "likelihood is not finite");
    int nt = L->nt;
    double sum = 0;
    int cnt = 0, mx = 0;
    int64_t bytes = 0;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < i; ++j) {
            int r = L->h_ranks[(size_t)i * nt + j];
            sum += r;
            ++cnt;
            mx = std::max(mx, r);
            bytes += (int64_t)(tile_rows(n, L->nb, i) + tile_rows(n, L->nb, j)) * r * 8;
        }
    out->max_rank = mx;
    out->mean_rank = cnt ? sum / cnt : 0.0;
    out->offdiag_bytes = bytes;
    out->dense_bytes = (int64_t)nt * (nt - 1) / 2 * L->nb * L->nb * 8;
    out->flops = st.flops;
}

// One evaluation on one precision path (df: the mixed path's products in
// paired FP32; tc: those products on the tensor cores).
static void loglik_once(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, tlr_theta theta,
                        const tlr_opts *opts, tlr_mat *L, tlr_result *out, cudaStream_t s, bool df,
                        bool tc = false) {
    MaternParams P = params_of(theta);
    std::memset(out, 0, sizeof *out);
    out->info = -1;
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_a, s));
    build_matern_table(&P, ctx->d_mtab, s);
    status_reset(ctx, s);
    FactorStats st;
    long long inf = -1;
    DevBuf acc(3 * sizeof(double), s), y((size_t)n * sizeof(double), s);
    TLR_CUDA_TRY(cudaMemsetAsync(acc.as<double>(), 0, 3 * sizeof(double), s));
    out->precision_used = tc ? TLR_PREC_TENSOR : (df ? TLR_PREC_MIXED : TLR_PREC_FP64);
    try {
        factor(ctx, s, L, FactorMode::Matern, xy, &P, opts->eps * theta.sigma2, &st, &inf, z,
               y.as<double>(), acc.as<double>(), df, tc);
    } catch (const Error &) {
        out->info = inf;
        throw;
    }
    double h[3];
    TLR_CUDA_TRY(cudaMemcpyAsync(h, acc.as<double>(), sizeof h, cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_b, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    long long sinfo = -1;
    int sc = status_fetch(ctx, s, &sinfo);
    if (sc) {
        out->info = sinfo;
        throw make_error(sc, "likelihood: device status %d (info %lld)", sc, sinfo);
    }
    fill_result(out, n, L, h, st);
    float ms = 0.f;
    TLR_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b));
    out->ms_total = ms;
    ctx->last_gemm_ms = st.gemm_ms;
    ctx->last_gemm_flops = st.gemm_flops;
    ctx->last_matern_entries = st.matern_entries;
    ctx->last_panel_launches = st.panel_launches;
    for (int k = 0; k < kStages; ++k) ctx->last_stage_ms[k] = st.stage_ms[k];
    for (int k = 0; k < kDetail; ++k) ctx->last_detail_ms[k] = st.detail_ms[k];
}

static void loglik_impl(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, tlr_theta theta,
                        const tlr_opts *opts, tlr_mat *L, tlr_result *out, cudaStream_t s) {
    check_arg(xy && z && opts && L && out, "xy/z/opts/L/out");
    check_arg(n > 0 && L->n == n && L->nb == opts->nb, "L does not match n/nb");
    check_arg(opts->eps >= 0 && std::isfinite(opts->eps), "eps");
    check_arg(opts->precision == TLR_PREC_FP64 || opts->precision == TLR_PREC_MIXED ||
                  opts->precision == TLR_PREC_AUTO || opts->precision == TLR_PREC_TENSOR, "precision");
    if (opts->precision == TLR_PREC_TENSOR && !tc_available())
        throw make_error(TLR_ERR_CUDA, "TLR_PREC_TENSOR needs an sm_103a device");
    if (opts->precision != TLR_PREC_AUTO) {
        loglik_once(ctx, xy, z, n, theta, opts, L, out, s, opts->precision != TLR_PREC_FP64,
                    opts->precision == TLR_PREC_TENSOR);
        L->last_pivot2 = out->min_pivot2 / theta.sigma2;
        return;
    }
    // auto: FP64 at once if the previous likelihood on this matrix found an
    // ill-conditioned covariance; otherwise the mixed path, and the FP64 path
    // again, from the same starting rank map, if this factor shows one (or
    // the mixed factorisation met a non-positive pivot)
    const std::vector<int32_t> hint = L->h_ranks;
    float ms_mixed = 0.f;
    const bool predict64 = L->last_pivot2 > 0.0 && L->last_pivot2 < TLR_AUTO_PIVOT2;
    if (!predict64) {
        try {
            loglik_once(ctx, xy, z, n, theta, opts, L, out, s, true);
            L->last_pivot2 = out->min_pivot2 / theta.sigma2;
            if (L->last_pivot2 >= TLR_AUTO_PIVOT2) return;
            ms_mixed = out->ms_total;
        } catch (const Error &e) {
            if (e.code != TLR_ERR_NOT_SPD) throw;
            TLR_CUDA_TRY(cudaStreamSynchronize(s));
        }
        L->h_ranks = hint;
    }
    loglik_once(ctx, xy, z, n, theta, opts, L, out, s, false);
    L->last_pivot2 = out->min_pivot2 / theta.sigma2;
    out->ms_total += ms_mixed;
}

static bool per_entry_error(int code) {
    return code == TLR_ERR_NOT_SPD || code == TLR_ERR_RANK || code == TLR_ERR_NAN;
}

// The entries es on one precision path, their factorisations in lockstep
// (factor_group).  A single entry takes loglik_once.  Failures that belong
// to one entry (NOT_SPD, RANK, NAN) go to its status; others throw.  Each
// entry's ms_total is the device time of the whole call.
static void loglik_group_once(tlr_ctx *ctx, const std::vector<BatchEntry *> &es, cudaStream_t s, bool df, bool tc) {
    const int G = (int)es.size();
    if (G == 0) return;
    if (G == 1) {
        BatchEntry &e = *es[0];
        try {
            loglik_once(ctx, e.xy, e.z, e.n, e.theta, e.opts, e.L, e.out, s, df, tc);
            e.status = TLR_OK;
        } catch (const Error &err) {
            if (!per_entry_error(err.code)) throw;
            e.status = err.code;
            e.msg = err.msg;
        }
        return;
    }
    const int cnt = kTabIntervals * kTabCoef;
    std::vector<MaternParams> P(G);
    std::vector<FactorStats> st(G);
    std::vector<long long> info(G, -1);
    int64_t ntot = 0;
    for (BatchEntry *e : es) ntot += e->n;
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_a, s));
    DevBuf tabs((size_t)G * 2 * cnt * sizeof(double), s);
    DevBuf acc((size_t)G * 3 * sizeof(double), s), y((size_t)ntot * sizeof(double), s);
    TLR_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, (size_t)(G + 1) * sizeof(DevStatus), s));
    TLR_CUDA_TRY(cudaMemsetAsync(acc.as<double>(), 0, (size_t)G * 3 * sizeof(double), s));
    std::vector<FactorItem> items(G);
    int64_t yoff = 0;
    for (int g = 0; g < G; ++g) {
        BatchEntry &e = *es[(size_t)g];
        std::memset(e.out, 0, sizeof *e.out);
        e.out->info = -1;
        e.out->precision_used = tc ? TLR_PREC_TENSOR : (df ? TLR_PREC_MIXED : TLR_PREC_FP64);
        P[(size_t)g] = params_of(e.theta);
        build_matern_table(&P[(size_t)g], tabs.as<double>() + (size_t)g * 2 * cnt, s);
        FactorItem &F = items[(size_t)g];
        F.M = e.L;
        F.xy = e.xy;
        F.P = &P[(size_t)g];
        F.tau = e.opts->eps * e.theta.sigma2;
        F.stats = &st[(size_t)g];
        F.info = &info[(size_t)g];
        F.z = e.z;
        F.y = y.as<double>() + yoff;
        F.acc = acc.as<double>() + 3 * g;
        yoff += e.n;
    }
    factor_group(ctx, s, items, FactorMode::Matern, df, tc);
    std::vector<double> h((size_t)G * 3);
    TLR_CUDA_TRY(cudaMemcpyAsync(h.data(), acc.as<double>(), h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_b, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    TLR_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b));
    for (int g = 0; g < G; ++g) {
        BatchEntry &e = *es[(size_t)g];
        const FactorItem &F = items[(size_t)g];
        e.out->ms_total = ms;
        if (F.err != TLR_OK) {
            e.status = F.err;
            e.msg = F.msg;
            e.out->info = info[(size_t)g];
            continue;
        }
        try {
            fill_result(e.out, e.n, e.L, h.data() + 3 * g, st[(size_t)g]);
            e.status = TLR_OK;
        } catch (const Error &err) {
            e.status = err.code;
            e.msg = err.msg;
        }
    }
    ctx->last_gemm_ms = st[0].gemm_ms;
    ctx->last_gemm_flops = st[0].gemm_flops;
    ctx->last_matern_entries = st[0].matern_entries;
    ctx->last_panel_launches = st[0].panel_launches;
    for (int k = 0; k < kStages; ++k) ctx->last_stage_ms[k] = st[0].stage_ms[k];
    for (int k = 0; k < kDetail; ++k) ctx->last_detail_ms[k] = st[0].detail_ms[k];
}

// The precision logic of loglik_impl over a batch: every entry computes what
// tlr_loglik would compute for it alone (the same path choices, from the same
// rank map); the entries of one path run as one group.
static void loglik_group(tlr_ctx *ctx, std::vector<BatchEntry> &es, cudaStream_t s) {
    const int prec = es[0].opts->precision;
    if (prec == TLR_PREC_TENSOR && !tc_available())
        throw make_error(TLR_ERR_CUDA, "TLR_PREC_TENSOR needs an sm_103a device");
    std::vector<BatchEntry *> all;
    for (BatchEntry &e : es) all.push_back(&e);
    if (prec != TLR_PREC_AUTO) {
        loglik_group_once(ctx, all, s, prec != TLR_PREC_FP64, prec == TLR_PREC_TENSOR);
        for (BatchEntry *e : all)
            if (e->status == TLR_OK) e->L->last_pivot2 = e->out->min_pivot2 / e->theta.sigma2;
        return;
    }
    std::vector<std::vector<int32_t>> hint(es.size());
    std::vector<float> ms_mixed(es.size(), 0.f);
    std::vector<BatchEntry *> mixed, fp64;
    for (size_t q = 0; q < es.size(); ++q) {
        hint[q] = es[q].L->h_ranks;
        const double p2 = es[q].L->last_pivot2;
        (p2 > 0.0 && p2 < TLR_AUTO_PIVOT2 ? fp64 : mixed).push_back(&es[q]);
    }
    loglik_group_once(ctx, mixed, s, true, false);
    for (BatchEntry *e : mixed) {
        const size_t q = (size_t)(e - es.data());
        if (e->status == TLR_OK) {
            e->L->last_pivot2 = e->out->min_pivot2 / e->theta.sigma2;
            if (e->L->last_pivot2 >= TLR_AUTO_PIVOT2) continue;
            ms_mixed[q] = e->out->ms_total;
        } else if (e->status != TLR_ERR_NOT_SPD) {
            continue;
        }
        e->L->h_ranks = hint[q];
        fp64.push_back(e);
    }
    std::sort(fp64.begin(), fp64.end());  // entry order
    loglik_group_once(ctx, fp64, s, false, false);
    for (BatchEntry *e : fp64) {
        const size_t q = (size_t)(e - es.data());
        if (e->status == TLR_OK) e->L->last_pivot2 = e->out->min_pivot2 / e->theta.sigma2;
        e->out->ms_total += ms_mixed[q];
    }
}

}  // extern "C"

void tlr::loglik_batch(tlr_ctx *ctx, std::vector<BatchEntry> &es, cudaStream_t s) {
    const int count = (int)es.size();
    check_arg(count >= 1 && count <= kMaxGroup, "count must be 1..32");
    for (int g = 0; g < count; ++g) {
        const BatchEntry &e = es[(size_t)g];
        const tlr_opts *o = e.opts;
        check_arg(e.xy && e.z && e.L && e.opts && e.out, "xy[g]/z[g]/L[g]/opts/out");
        check_arg(e.n > 0 && e.L->n == e.n && e.L->nb == o->nb, "L[g] does not match n[g]/nb");
        check_arg(o->eps >= 0 && std::isfinite(o->eps), "eps");
        check_arg(o->precision == es[0].opts->precision, "one precision for all entries");
        check_arg(o->precision == TLR_PREC_FP64 || o->precision == TLR_PREC_MIXED || o->precision == TLR_PREC_AUTO ||
                      o->precision == TLR_PREC_TENSOR, "precision");
        for (int h = 0; h < g; ++h) check_arg(es[(size_t)h].L != e.L, "every entry needs its own L");
    }
    loglik_group(ctx, es, s);
}

extern "C" {

int tlr_loglik_batch(tlr_ctx *ctx, int count, const double *const *xy, const double *const *z, const int64_t *n,
                     const tlr_theta *theta, const tlr_opts *opts, tlr_mat *const *L, tlr_result *out, int *status,
                     void *stream) {
    std::vector<BatchEntry> es;
    int rc = guarded(ctx, [&] {
        check_arg(count >= 1 && count <= kMaxGroup, "count must be 1..32");
        check_arg(xy && z && n && theta && opts && L && out, "xy/z/n/theta/opts/L/out");
        for (int g = 0; g < count; ++g) {
            BatchEntry e{};
            e.xy = xy[g];
            e.z = z[g];
            e.n = n[g];
            e.theta = theta[g];
            e.opts = opts + g;
            e.L = L[g];
            e.out = out + g;
            es.push_back(e);
        }
        loglik_batch(ctx, es, (cudaStream_t)stream);
    });
    if (rc != TLR_OK) {
        if (status)
            for (int g = 0; g < count; ++g) status[g] = rc;
        return rc;
    }
    int first = TLR_OK;
    for (int g = 0; g < count; ++g) {
        if (status) status[g] = es[(size_t)g].status;
        if (es[(size_t)g].status != TLR_OK && first == TLR_OK) {
            first = es[(size_t)g].status;
            ctx->err = es[(size_t)g].msg;
        }
    }
    return first;
}

int tlr_loglik(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, tlr_theta theta,
               const tlr_opts *opts, tlr_mat *L, tlr_result *out, void *stream) {
    return guarded(ctx, [&] { loglik_impl(ctx, xy, z, n, theta, opts, L, out, (cudaStream_t)stream); });
}

int tlr_loglik_host(tlr_ctx *ctx, const double *xy_host, const double *z_host, int64_t n, int order, uint64_t seed,
                    tlr_theta theta, const tlr_opts *opts, tlr_mat *L, tlr_result *out, void *stream) {
    return guarded(ctx, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        check_arg(xy_host && z_host && n > 0 && n < ((int64_t)1 << 31), "xy_host/z_host/n");
        check_arg(order >= TLR_ORDER_IDENTITY && order <= TLR_ORDER_MAXMIN, "order");
        // device copies of the inputs, the ordering and the ordered inputs
        DevBuf xy(2 * (size_t)n * sizeof(double), s), z((size_t)n * sizeof(double), s);
        DevBuf perm((size_t)n * sizeof(int64_t), s), xyo(2 * (size_t)n * sizeof(double), s),
            zo((size_t)n * sizeof(double), s);
        TLR_CUDA_TRY(cudaMemcpyAsync(xy.as<double>(), xy_host, 2 * (size_t)n * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        TLR_CUDA_TRY(cudaMemcpyAsync(z.as<double>(), z_host, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
        const double *x = xy.as<double>();
        int64_t *p = perm.as<int64_t>();
        switch (order) {
        case TLR_ORDER_IDENTITY: order_identity(n, p, s); break;
        case TLR_ORDER_RANDOM:
        case TLR_ORDER_MORTON:
        case TLR_ORDER_HILBERT: order_sfc(x, n, order, seed, p, nullptr, s); break;
        case TLR_ORDER_KDTREE: order_kdtree(x, n, p, s); break;
        case TLR_ORDER_MAXMIN: order_maxmin(x, n, p, s, ctx->num_sms); break;
        }
        permute_xy(x, p, n, 0, xyo.as<double>(), s);
        gather(p, z.as<double>(), n, zo.as<double>(), s);
        loglik_impl(ctx, xyo.as<double>(), zo.as<double>(), n, theta, opts, L, out, s);
    });
}

int tlr_profile(tlr_ctx *ctx, int enable, double *gemm_ms, double *gemm_flops, double *matern_entries,
                int *panel_launches) {
    if (!ctx) return TLR_ERR_ARG;
    ctx->profile = enable != 0;
    if (gemm_ms) *gemm_ms = ctx->last_gemm_ms;
    if (gemm_flops) *gemm_flops = ctx->last_gemm_flops;
    if (matern_entries) *matern_entries = ctx->last_matern_entries;
    if (panel_launches) *panel_launches = ctx->last_panel_launches;
    return TLR_OK;
}

int tlr_stage_times(tlr_ctx *ctx, double *ms) {
    if (!ctx || !ms) return TLR_ERR_ARG;
    for (int k = 0; k < kStages; ++k) ms[k] = ctx->last_stage_ms[k];
    return TLR_OK;
}

int tlr_detail_times(tlr_ctx *ctx, double *ms, int count) {
    if (!ctx || !ms || count < 0) return TLR_ERR_ARG;
    for (int k = 0; k < count && k < kDetail; ++k) ms[k] = ctx->last_detail_ms[k];
    return std::min(count, (int)kDetail);
}

int tlr_compress_times(tlr_ctx *ctx, double *ms) {
    if (!ctx || !ms) return TLR_ERR_ARG;
    for (int k = 0; k < 7; ++k) ms[k] = ctx->comp_ms[k];
    return TLR_OK;
}

int tlr_kernel_stats(tlr_ctx *ctx, double *out) {
    if (!ctx || !out) return TLR_ERR_ARG;
    out[0] = ctx->k16_ms;
    out[1] = ctx->k16_flops;
    out[2] = (double)ctx->k16_launches;
    out[3] = (double)ctx->k16_clusters;
    return TLR_OK;
}

int tlr_compress_stats(tlr_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return TLR_ERR_ARG;
    for (int k = 0; k < 7; ++k) out[k] = ctx->comp_stats[k];
    return TLR_OK;
}

int tlr_mle(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, const tlr_opts *opts,
            tlr_theta theta0, tlr_theta lo, tlr_theta hi, double tol, int max_iter, tlr_mat *L,
            tlr_theta *theta_hat, double *ll_hat, int *iters, void *stream) {
    return guarded(ctx, [&] {
        check_arg(theta_hat && ll_hat && iters && max_iter > 0 && tol > 0, "mle outputs");
        check_arg(mle_bounds_ok(lo, hi), "bounds");
        cudaStream_t s = (cudaStream_t)stream;
        // f = -l(theta); failed evaluations are +inf
        auto f = [&](tlr_theta th) -> double {
            tlr_result r;
            try {
                loglik_impl(ctx, xy, z, n, th, opts, L, &r, s);
            } catch (const Error &e) {
                if (e.code == TLR_ERR_NOT_SPD || e.code == TLR_ERR_RANK || e.code == TLR_ERR_NAN) {
                    cudaStreamSynchronize(s);
                    return INFINITY;
                }
                throw;
            }
            return -r.loglik;
        };
        mle_nelder_mead(f, theta0, lo, hi, tol, max_iter, theta_hat, ll_hat, iters);
    });
}

}  // extern "C"

// Dense FP64 tile kernels of the TLR Cholesky (Sec. 2; the diagonal tiles stay
// dense): blocked right-looking Cholesky of one diagonal tile, forward
// substitution with many right-hand sides, and the log-determinant /
// quadratic-form reductions of Eq. 1.2.
//
// Blocks of 32 rows/columns are factored or solved by one CTA in shared
// memory; everything else is a batched GEMM update so that it spreads over
// the whole GPU (one SM's FP64 pipe alone would take milliseconds per tile).
#include "common.cuh"
#include "dense.cuh"
#include "gemm.cuh"

namespace tlr {

constexpr int kBlk = 32;
constexpr int kStrip = 64;  // column strips of the trailing update

// Cholesky of the w x w diagonal block at (p0, p0) of A (lower part).
__global__ void k_potrf_block(double *__restrict__ A, int lda, int m, int p0, DevStatus *st,
                              long long row_base) {
    __shared__ double S[kBlk][kBlk + 1];
    __shared__ int bad;
    if (st->code) return;
    const int r = threadIdx.x;  // 32 threads
    const int w = min(kBlk, m - p0);
    double *B = A + (int64_t)p0 * lda + p0;
    for (int c = 0; c < w; ++c) S[r][c] = (r < w) ? B[(int64_t)c * lda + r] : 0.0;
    if (r == 0) bad = -1;
    __syncthreads();
    for (int c = 0; c < w; ++c) {
        if (r == c) {
            double d = S[c][c];
            if (!(d > 0.0)) bad = c;
            else S[c][c] = sqrt(d);
        }
        __syncthreads();
        if (bad >= 0) break;
        if (r > c && r < w) S[r][c] /= S[c][c];
        __syncthreads();
        if (r > c && r < w) {
            double lrc = S[r][c];
            for (int cc = c + 1; cc <= r; ++cc) S[r][cc] -= lrc * S[cc][c];
        }
        __syncthreads();
    }
    if (bad >= 0) {
        if (r == 0) set_status(st, TLR_ERR_NOT_SPD, row_base + p0 + bad);
        return;
    }
    if (r < w)
        for (int c = 0; c <= r; ++c) B[(int64_t)c * lda + r] = S[r][c];
}

// A[r, p0:p0+w] <- A[r, p0:p0+w] L^-T for rows p0+w <= r < m (one thread per row).
__global__ void k_trsm_right_lt(double *__restrict__ A, int lda, int m, int p0, const DevStatus *st) {
    __shared__ double L[kBlk][kBlk + 1];
    if (st->code) return;
    const int w = min(kBlk, m - p0);
    const double *Lb = A + (int64_t)p0 * lda + p0;
    for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        int rr = e % kBlk, cc = e / kBlk;
        L[rr][cc] = (rr < w && cc < w && cc <= rr) ? Lb[(int64_t)cc * lda + rr] : 0.0;
    }
    __syncthreads();
    int r = p0 + w + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double x[kBlk];
    double *row = A + (int64_t)p0 * lda + r;
#pragma unroll
    for (int c = 0; c < kBlk; ++c) {
        if (c < w) {
            double a = row[(int64_t)c * lda];
#pragma unroll
            for (int k = 0; k < c; ++k) a -= x[k] * L[c][k];
            x[c] = a / L[c][c];
        } else {
            x[c] = 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
        if (c < w) row[(int64_t)c * lda] = x[c];
}

__global__ void k_zero_upper(double *__restrict__ A, int lda, int m) {
    int c = blockIdx.x;
    for (int r = threadIdx.x; r < c && c < m; r += blockDim.x) A[(int64_t)c * lda + r] = 0.0;
}

void potrf_dense(tlr_ctx *ctx, cudaStream_t s, double *A, int lda, int m, long long row_base) {
    for (int p0 = 0; p0 < m; p0 += kBlk) {
        int w = std::min(kBlk, m - p0);
        launch(k_potrf_block, 1, kBlk, 0, s, A, lda, m, p0, ctx->d_status, row_base);
        int rest = m - p0 - w;
        if (rest <= 0) break;
        launch(k_trsm_right_lt, (unsigned)ceil_div(rest, 128), 128, 0, s, A, lda, m, p0, ctx->d_status);
        TLR_CHECK_LAUNCH();
        // trailing lower update A22 -= P P', one problem per 64-column strip
        double *P = A + (int64_t)p0 * lda + p0 + w;
        double *A22 = A + (int64_t)(p0 + w) * lda + p0 + w;
        std::vector<GemmProb> probs;
        for (int cb = 0; cb < rest; cb += kStrip) {
            GemmProb g{};
            g.A = P + cb;
            g.B = P + cb;
            g.C = A22 + (int64_t)cb * lda + cb;
            g.m = rest - cb;
            g.n = std::min(kStrip, rest - cb);
            g.k = w;
            g.lda = lda;
            g.ldb = lda;
            g.ldc = lda;
            probs.push_back(g);
        }
        gemm_batched(ctx, s, false, true, probs, -1.0, 1.0);
    }
    launch(k_zero_upper, m, 128, 0, s, A, lda, m);
    TLR_CHECK_LAUNCH();
}

// Solve L X = B for the 32-row block at p0 of every right-hand side column.
// Columns of all problems are concatenated; col_off gives each problem's start.
__global__ void k_trsm_left_block(const double *__restrict__ Lm, int ldl, int m, int p0,
                                  const RhsDesc *__restrict__ rhs, const int *__restrict__ col_off,
                                  int nrhs, const DevStatus *st) {
    __shared__ double L[kBlk][kBlk + 1];
    if (st->code) return;
    const int w = min(kBlk, m - p0);
    const double *Lb = Lm + (int64_t)p0 * ldl + p0;
    for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
        int rr = e % kBlk, cc = e / kBlk;
        L[rr][cc] = (rr < w && cc < w && cc <= rr) ? Lb[(int64_t)cc * ldl + rr] : 0.0;
    }
    __syncthreads();
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= col_off[nrhs]) return;
    int lo = 0, hi = nrhs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (col_off[mid] <= col) lo = mid; else hi = mid - 1;
    }
    const RhsDesc d = rhs[lo];
    double *b = d.B + (int64_t)(col - col_off[lo]) * d.ld + p0;
    double x[kBlk];
#pragma unroll
    for (int r = 0; r < kBlk; ++r) {
        if (r < w) {
            double a = b[r];
#pragma unroll
            for (int k = 0; k < r; ++k) a -= L[r][k] * x[k];
            x[r] = a / L[r][r];
        } else {
            x[r] = 0.0;
        }
    }
#pragma unroll
    for (int r = 0; r < kBlk; ++r)
        if (r < w) b[r] = x[r];
}

void trsm_left_lower(tlr_ctx *ctx, cudaStream_t s, const double *L, int ldl, int m,
                     const std::vector<RhsDesc> &rhs) {
    std::vector<RhsDesc> act;
    for (const RhsDesc &d : rhs)
        if (d.ncols > 0) act.push_back(d);
    if (act.empty() || m <= 0) return;
    std::vector<int> off(act.size() + 1, 0);
    for (size_t b = 0; b < act.size(); ++b) off[b + 1] = off[b] + act[b].ncols;
    auto *dr = (const RhsDesc *)stage_push(ctx, act.data(), act.size() * sizeof(RhsDesc), s);
    auto *doff = (const int *)stage_push(ctx, off.data(), off.size() * sizeof(int), s);
    int total = off.back();
    for (int p0 = 0; p0 < m; p0 += kBlk) {
        int w = std::min(kBlk, m - p0);
        launch(k_trsm_left_block, (unsigned)ceil_div(total, 128), 128, 0, s, L, ldl, m, p0, dr, doff,
                                                                         (int)act.size(), ctx->d_status);
        TLR_CHECK_LAUNCH();
        int rest = m - p0 - w;
        if (rest <= 0) break;
        std::vector<GemmProb> probs;
        for (const RhsDesc &d : act) {
            GemmProb g{};
            g.A = L + (int64_t)p0 * ldl + p0 + w;
            g.B = d.B + p0;
            g.C = d.B + p0 + w;
            g.m = rest;
            g.n = d.ncols;
            g.k = w;
            g.lda = ldl;
            g.ldb = d.ld;
            g.ldc = d.ld;
            probs.push_back(g);
        }
        gemm_batched(ctx, s, false, false, probs, -1.0, 1.0);
    }
}

// acc[0] += sum_r log A[r, r]  (one block, fixed reduction order)
__global__ void k_diag_logsum(const double *__restrict__ A, int lda, int m, double *acc,
                              const DevStatus *st) {
    __shared__ double part[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += log(A[(int64_t)r * lda + r]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0 && !st->code) acc[0] += part[0];
}

// acc[0] += sum v_r^2 (one block, fixed reduction order)
__global__ void k_sumsq(const double *__restrict__ v, int m, double *acc) {
    __shared__ double part[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += v[r] * v[r];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) acc[0] += part[0];
}

void diag_logsum(cudaStream_t s, const double *A, int lda, int m, double *acc, const DevStatus *st) {
    launch(k_diag_logsum, 1, 256, 0, s, A, lda, m, acc, st);
    TLR_CHECK_LAUNCH();
}

void sumsq(cudaStream_t s, const double *v, int m, double *acc) {
    launch(k_sumsq, 1, 256, 0, s, v, m, acc);
    TLR_CHECK_LAUNCH();
}

}  // namespace tlr

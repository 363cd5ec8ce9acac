// Batched FP64 GEMM with per-problem sizes and a pluggable epilogue.
//
// C_b = epilogue(alpha * op(A_b) op(B_b), C_b) for every problem b of a batch;
// one launch covers all problems (blockIdx.x runs over the concatenated
// 64 x 64 output tiles; a binary search over the per-problem tile offsets
// finds the problem).  Matrices are column major.  Each thread accumulates a
// 4 x 4 block over K in steps of 16 staged through shared memory.  GB300's
// FP64 pipe issues 2 DFMA/clk/SM, so this register blocking already keeps the
// kernel bound by the FP64 units, not by shared memory or HBM.
#pragma once

#include "common.cuh"
#include "matern.cuh"

namespace tlr {

struct GemmProb {
    const double *A;
    const double *B;
    double *C;
    int m, n, k;
    int lda, ldb, ldc;
    int64_t ri0, ci0;  // epilogue data: first global row / column index
};

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

// C = alpha * AB + beta * C   (C is not read when beta == 0)
struct EpiLinear {
    double beta;
    __device__ __forceinline__ double operator()(const GemmProb &, int, int, double ab,
                                                 const double *c) const {
        return beta == 0.0 ? ab : ab + beta * (*c);
    }
};

// C = Sigma(row point, col point) + alpha * AB; rows/cols past n give 0.
struct EpiMatern {
    const double *xy;
    int64_t n;
    MaternParams P;
    __device__ __forceinline__ double operator()(const GemmProb &p, int r, int c, double ab,
                                                 const double *) const {
        int64_t gr = p.ri0 + r, gc = p.ci0 + c;
        if (gr >= n || gc >= n) return 0.0;
        return matern_cov(xy[gr], xy[n + gr], xy[gc], xy[n + gc], P) + ab;
    }
};

template <bool TA, bool TB, class Epi>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_f64(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob,
           double alpha, Epi epi) {
    __shared__ double As[kGemmBK][kGemmBM + 1];
    __shared__ double Bs[kGemmBK][kGemmBN + 1];
    const int tid = threadIdx.x;
    // locate the problem
    int lo = 0, hi = nprob - 1, t = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmProb p = probs[lo];
    int local = t - tile_off[lo];
    int tm = (p.m + kGemmBM - 1) / kGemmBM;
    if (tm == 0) return;
    const int m0 = (local % tm) * kGemmBM, n0 = (local / tm) * kGemmBN;
    const int r0 = (tid & 15) * 4, c0 = (tid >> 4) * 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int k0 = 0; k0 < p.k; k0 += kGemmBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int r, kk;
            if (!TA) { r = tid & 63; kk = (tid >> 6) + 4 * q; }
            else     { kk = tid & 15; r = (tid >> 4) + 16 * q; }
            int gr = m0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gr < p.m && gk < p.k)
                v = TA ? p.A[(int64_t)gr * p.lda + gk] : p.A[(int64_t)gk * p.lda + gr];
            As[kk][r] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c, kk;
            if (!TB) { kk = tid & 15; c = (tid >> 4) + 16 * q; }
            else     { c = tid & 63; kk = (tid >> 6) + 4 * q; }
            int gc = n0 + c, gk = k0 + kk;
            double v = 0.0;
            if (gc < p.n && gk < p.k)
                v = TB ? p.B[(int64_t)gk * p.ldb + gc] : p.B[(int64_t)gc * p.ldb + gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmBK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][r0 + q]; b[q] = Bs[kk][c0 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        int c = n0 + c0 + y;
        if (c >= p.n) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            int r = m0 + r0 + x;
            if (r >= p.m) continue;
            double *cp = p.C + (int64_t)c * p.ldc + r;
            *cp = epi(p, r, c, alpha * acc[x][y], cp);
        }
    }
}

// Host launcher: uploads the descriptors through the context's staging
// buffers and launches one kernel for the whole batch.
void gemm_batched(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                  double alpha, double beta);
void gemm_batched_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs,
                         double alpha, const double *xy, int64_t n, const MaternParams &P);

}  // namespace tlr

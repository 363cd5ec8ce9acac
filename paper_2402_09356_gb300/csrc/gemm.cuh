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
    const float2 *A2;  // paired-FP32 copies of A and B (same layout), for k_gemm_df
    const float2 *B2;
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

// The same product with paired-FP32 ("double-float") arithmetic on the FP32
// pipe, which GB300 issues 64 times faster than FP64.  Each operand x is read
// as hi = fl32(x), lo = fl32(x - hi) (|x - hi - lo| <= 2^-48 |x|) from the
// copies A2, B2 that split_f2 made once per operand.  A product is a_hi b_hi + (its exact rounding error,
// by FMA) + a_hi b_lo + a_lo b_hi; the high parts are accumulated with TwoSum
// (Knuth; Dekker 1971) and all low-order terms in a second FP32 accumulator,
// so a K-term dot product carries about 46 bits, i.e. ~1e-13 relative error.
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float &ch, float &cl) {
    float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float sum = __fadd_rn(ch, p);
    float bp = __fsub_rn(sum, ch);
    float err = __fadd_rn(__fsub_rn(ch, __fsub_rn(sum, bp)), __fsub_rn(p, bp));
    ch = sum;
    cl = __fadd_rn(cl, __fadd_rn(err, e));
}

template <bool TA, bool TB, class Epi>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_df(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob, double alpha,
          Epi epi) {
    __shared__ float2 As[kGemmBK][kGemmBM + 1];
    __shared__ float2 Bs[kGemmBK][kGemmBN + 1];
    const int tid = threadIdx.x;
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
    float ch[4][4], cl[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { ch[a][b] = 0.f; cl[a][b] = 0.f; }
    for (int k0 = 0; k0 < p.k; k0 += kGemmBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int r, kk;
            if (!TA) { r = tid & 63; kk = (tid >> 6) + 4 * q; }
            else     { kk = tid & 15; r = (tid >> 4) + 16 * q; }
            int gr = m0 + r, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gr < p.m && gk < p.k)
                v = TA ? p.A2[(int64_t)gr * p.lda + gk] : p.A2[(int64_t)gk * p.lda + gr];
            As[kk][r] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c, kk;
            if (!TB) { kk = tid & 15; c = (tid >> 4) + 16 * q; }
            else     { c = tid & 63; kk = (tid >> 6) + 4 * q; }
            int gc = n0 + c, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gc < p.n && gk < p.k)
                v = TB ? p.B2[(int64_t)gk * p.ldb + gc] : p.B2[(int64_t)gc * p.ldb + gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmBK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][r0 + q]; b[q] = Bs[kk][c0 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) df_fma(a[x].x, a[x].y, b[y].x, b[y].y, ch[x][y], cl[x][y]);
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
            *cp = epi(p, r, c, alpha * ((double)ch[x][y] + (double)cl[x][y]), cp);
        }
    }
}

// Host launcher: uploads the descriptors through the context's staging
// buffers and launches one kernel for the whole batch.
// dst[j * ld + i] = (hi, lo) of src[j * ld + i] for an m x n column-major block.
void split_f2(cudaStream_t s, const double *src, int ld, int m, int n, float2 *dst);

struct SplitDesc {
    const double *src;
    float2 *dst;  // same leading dimension as src
    int ld, m, n;
};
// split_f2 for a batch of blocks in one launch.
void split_f2_batched(tlr_ctx *ctx, cudaStream_t s, const std::vector<SplitDesc> &descs);

// df = true selects the paired-FP32 kernel (FP64-accurate products on the FP32
// pipe); every problem must then carry A2/B2 copies made by split_f2.
void gemm_batched(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                  double alpha, double beta, bool df = false);
void gemm_batched_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs,
                         double alpha, const double *xy, int64_t n, const MaternParams &P, bool df = false);

}  // namespace tlr

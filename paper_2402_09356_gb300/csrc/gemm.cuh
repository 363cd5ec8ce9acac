// Batched FP64 GEMM with per-problem sizes and a pluggable epilogue.
//
// C_b = epilogue(alpha * op(A_b) op(B_b), C_b) for every problem b of a batch;
// one launch covers all problems of one tile shape (blockIdx.x runs over the
// concatenated output tiles; a binary search over the per-problem tile
// offsets finds the problem).  Matrices are column major.  Each thread
// accumulates a register block over K in steps of 16 staged through shared
// memory.  GB300's FP64 pipe issues 2 DFMA/clk/SM, so this register blocking
// already keeps the kernel bound by the FP64 units, not by shared memory or
// HBM.
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
    int item;          // EpiMaternMulti: the factorisation whose covariance the problem holds
};

constexpr int kGemmBK = 16, kGemmThreads = 256;

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

// The Matern epilogue for the panels of several factorisations in one
// launch: problem p takes its locations and parameters from items[p.item]
// (the same arithmetic as EpiMatern).
struct MaternItem {
    const double *xy;
    int64_t n;
    MaternParams P;
};
struct EpiMaternMulti {
    const MaternItem *items;
    __device__ __forceinline__ double operator()(const GemmProb &p, int r, int c, double ab,
                                                 const double *) const {
        const MaternItem &it = items[p.item];
        const int64_t n = it.n, gr = p.ri0 + r, gc = p.ci0 + c;
        if (gr >= n || gc >= n) return 0.0;
        return matern_cov(it.xy[gr], it.xy[n + gr], it.xy[gc], it.xy[n + gc], it.P) + ab;
    }
};

// Locate the problem of output tile t (binary search over the per-problem
// tile offsets) and the tile's first row and column.
template <int BM, int BN>
__device__ __forceinline__ bool gemm_tile(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off,
                                          int nprob, int t, GemmProb &p, int &m0, int &n0) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    p = probs[lo];
    const int local = t - tile_off[lo];
    const int tm = (p.m + BM - 1) / BM;
    if (tm == 0) return false;
    m0 = (local % tm) * BM;
    n0 = (local / tm) * BN;
    return true;
}

// BM x BN output tiles, CTA b taking tiles b, b + gridDim.x, ... (a grid
// smaller than the tile count keeps the product to that many CTAs), 256
// threads per CTA (a 16 x 16 thread grid, BM/16 x BN/16 outputs per thread),
// K in steps of 16 through shared memory.
// Tiles of 64 x 64 serve large products; 32-row or 32-column tiles serve the
// many thin products of the low-rank updates (ranks of a few tens), whose
// padding would otherwise dominate.
template <int BM, int BN, bool TA, bool TB, class Epi>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_f64(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob, int ntiles,
           double alpha, Epi epi) {
    constexpr int TM = BM / 16, TN = BN / 16;
    __shared__ double As[kGemmBK][BM + 1];
    __shared__ double Bs[kGemmBK][BN + 1];
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    GemmProb p;
    int m0, n0;
    if (!gemm_tile<BM, BN>(probs, tile_off, nprob, t, p, m0, n0)) continue;
    const int r0 = (tid & 15) * TM, c0 = (tid >> 4) * TN;
    double acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = 0.0;

    for (int k0 = 0; k0 < p.k; k0 += kGemmBK) {
#pragma unroll
        for (int e = tid; e < BM * kGemmBK; e += kGemmThreads) {
            const int r = TA ? e / kGemmBK : e % BM, kk = TA ? e % kGemmBK : e / BM;
            const int gr = m0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gr < p.m && gk < p.k)
                v = TA ? p.A[(int64_t)gr * p.lda + gk] : p.A[(int64_t)gk * p.lda + gr];
            As[kk][r] = v;
        }
#pragma unroll
        for (int e = tid; e < BN * kGemmBK; e += kGemmThreads) {
            const int c = TB ? e % BN : e / kGemmBK, kk = TB ? e / BN : e % kGemmBK;
            const int gc = n0 + c, gk = k0 + kk;
            double v = 0.0;
            if (gc < p.n && gk < p.k)
                v = TB ? p.B[(int64_t)gk * p.ldb + gc] : p.B[(int64_t)gc * p.ldb + gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmBK; ++kk) {
            double a[TM], b[TN];
#pragma unroll
            for (int q = 0; q < TM; ++q) a[q] = As[kk][r0 + q];
#pragma unroll
            for (int q = 0; q < TN; ++q) b[q] = Bs[kk][c0 + q];
#pragma unroll
            for (int x = 0; x < TM; ++x)
#pragma unroll
                for (int y = 0; y < TN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < TN; ++y) {
        int c = n0 + c0 + y;
        if (c >= p.n) continue;
#pragma unroll
        for (int x = 0; x < TM; ++x) {
            int r = m0 + r0 + x;
            if (r >= p.m) continue;
            double *cp = p.C + (int64_t)c * p.ldc + r;
            *cp = epi(p, r, c, alpha * acc[x][y], cp);
        }
    }
    __syncthreads();  // the next tile reuses the shared tiles
    }
}

// The same product with paired-FP32 ("double-float") arithmetic on the FP32
// pipe, which GB300 issues 64 times faster than FP64.  Each operand x is read
// as hi = fl32(x), lo = fl32(x - hi) (|x - hi - lo| <= 2^-48 |x|) from the
// copies A2, B2 that split_f2 made once per operand.  A product is
// a_hi b_hi + (its exact rounding error, by FMA) + a_hi b_lo + a_lo b_hi; the
// high parts are accumulated with TwoSum (Knuth; Dekker 1971) and all
// low-order terms in a second FP32 accumulator, so a K-term dot product
// carries about 46 bits, i.e. ~1e-13 relative error.
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

template <int BM, int BN, bool TA, bool TB, class Epi>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_df(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob, int ntiles,
          double alpha, Epi epi) {
    constexpr int TM = BM / 16, TN = BN / 16;
    __shared__ float2 As[kGemmBK][BM + 1];
    __shared__ float2 Bs[kGemmBK][BN + 1];
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    GemmProb p;
    int m0, n0;
    if (!gemm_tile<BM, BN>(probs, tile_off, nprob, t, p, m0, n0)) continue;
    const int r0 = (tid & 15) * TM, c0 = (tid >> 4) * TN;
    float ch[TM][TN], cl[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) { ch[a][b] = 0.f; cl[a][b] = 0.f; }
    for (int k0 = 0; k0 < p.k; k0 += kGemmBK) {
#pragma unroll
        for (int e = tid; e < BM * kGemmBK; e += kGemmThreads) {
            const int r = TA ? e / kGemmBK : e % BM, kk = TA ? e % kGemmBK : e / BM;
            const int gr = m0 + r, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gr < p.m && gk < p.k)
                v = TA ? p.A2[(int64_t)gr * p.lda + gk] : p.A2[(int64_t)gk * p.lda + gr];
            As[kk][r] = v;
        }
#pragma unroll
        for (int e = tid; e < BN * kGemmBK; e += kGemmThreads) {
            const int c = TB ? e % BN : e / kGemmBK, kk = TB ? e / BN : e % kGemmBK;
            const int gc = n0 + c, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gc < p.n && gk < p.k)
                v = TB ? p.B2[(int64_t)gk * p.ldb + gc] : p.B2[(int64_t)gc * p.ldb + gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGemmBK; ++kk) {
            float2 a[TM], b[TN];
#pragma unroll
            for (int q = 0; q < TM; ++q) a[q] = As[kk][r0 + q];
#pragma unroll
            for (int q = 0; q < TN; ++q) b[q] = Bs[kk][c0 + q];
#pragma unroll
            for (int x = 0; x < TM; ++x)
#pragma unroll
                for (int y = 0; y < TN; ++y) df_fma(a[x].x, a[x].y, b[y].x, b[y].y, ch[x][y], cl[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < TN; ++y) {
        int c = n0 + c0 + y;
        if (c >= p.n) continue;
#pragma unroll
        for (int x = 0; x < TM; ++x) {
            int r = m0 + r0 + x;
            if (r >= p.m) continue;
            double *cp = p.C + (int64_t)c * p.ldc + r;
            *cp = epi(p, r, c, alpha * ((double)ch[x][y] + (double)cl[x][y]), cp);
        }
    }
    __syncthreads();  // the next tile reuses the shared tiles
    }
}

// Matrix-vector products (n = 1) with the linear epilogue:
//   TA:  one warp per output, lanes over k (the row of A' is contiguous);
//   !TA: one thread per output row, k in sequence (coalesced across threads).
// blockIdx.x runs over the concatenated per-problem tiles of kGemvRows outputs.
constexpr int kGemvRows = 256;
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads)
k_gemv(const GemmProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob, double alpha, EpiLinear epi) {
    int lo = 0, hi = nprob - 1, t = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmProb p = probs[lo];
    const int r0 = (t - tile_off[lo]) * kGemvRows;
    auto bk = [&](int k) { return TB ? p.B[(int64_t)k * p.ldb] : p.B[k]; };
    if (TA) {
        const int lane = threadIdx.x & 31;
        for (int r = r0 + (threadIdx.x >> 5); r < min(p.m, r0 + kGemvRows); r += kGemmThreads / 32) {
            const double *a = p.A + (int64_t)r * p.lda;
            double d = 0.0;
            for (int k = lane; k < p.k; k += 32) d = fma(a[k], bk(k), d);
#pragma unroll
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
            if (lane == 0) p.C[r] = epi(p, r, 0, alpha * d, p.C + r);
        }
    } else {
        const int r = r0 + threadIdx.x;
        if (r >= p.m) return;
        double d0 = 0.0, d1 = 0.0;
        int k = 0;
        for (; k + 1 < p.k; k += 2) {
            d0 = fma(p.A[(int64_t)k * p.lda + r], bk(k), d0);
            d1 = fma(p.A[(int64_t)(k + 1) * p.lda + r], bk(k + 1), d1);
        }
        if (k < p.k) d0 = fma(p.A[(int64_t)k * p.lda + r], bk(k), d0);
        p.C[r] = epi(p, r, 0, alpha * (d0 + d1), p.C + r);
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

// FP64, 32 x 32 output tiles for every problem: four times the CTAs of the
// 64 x 64 shape, for small square products on the critical path.
void gemm_batched_small(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                        double alpha, double beta);

// df = true selects the paired-FP32 kernel (FP64-accurate products on the FP32
// pipe); every problem must then carry A2/B2 copies made by split_f2.
void gemm_batched(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs,
                  double alpha, double beta, bool df = false);
// For a product running beside critical-path work: max_ctas > 0 caps the
// grid (the CTAs then loop over the tiles, one per SM); ctas_per_sm > 0
// allows at most that many of its CTAs on one SM.
void gemm_batched_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs,
                         double alpha, const double *xy, int64_t n, const MaternParams &P, bool df = false,
                         int max_ctas = 0, int ctas_per_sm = 0);
// The same for problems of several factorisations (problem b generates from
// items[b.item]; the table is copied to the device on s).
void gemm_batched_matern_multi(tlr_ctx *ctx, cudaStream_t s, const std::vector<GemmProb> &probs, double alpha,
                               const std::vector<MaternItem> &items, bool df, int ctas_per_sm = 0);

}  // namespace tlr

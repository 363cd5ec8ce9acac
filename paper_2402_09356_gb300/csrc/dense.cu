// Dense FP64 tile kernels of the TLR Cholesky (Sec. 2; the diagonal tiles stay
// dense): blocked right-looking Cholesky of one diagonal tile, forward
// substitution with many right-hand sides, and the log-determinant /
// quadratic-form reductions of Eq. 1.2.
//
// Blocks of 32 rows/columns are factored or solved by one CTA in shared
// memory; everything else is a batched GEMM update so that it spreads over
// the whole GPU (one SM's FP64 pipe alone would take milliseconds per tile).
#include <mutex>

#include <cooperative_groups.h>

#include "common.cuh"
#include "dense.cuh"
#include "ff.cuh"
#include "gemm.cuh"

namespace tlr {

namespace cg = cooperative_groups;

constexpr int kBlk = 32;


// ---------------------------------------------------------------------------
// Cholesky and inverse of one diagonal tile in a single launch.
//
// One cluster of kCl CTAs; the tile (m <= 1024, column major) stays in global
// memory, which for one tile is L2-resident, and every load goes to L2
// (__ldcg: another CTA may have written the line in an earlier phase).  A
// cluster barrier (release/acquire at cluster scope) separates dependent
// phases.  The factorisation and the inverse X = L^-1 advance together, in
// 32-wide block steps, two barriers a step.  Block step k:
//   1. (all CTAs) the panel rows below the block, A[r, k] <- A[r, k] L_kk^-T,
//      and the inverse's block row, X[k, :] <- L_kk^-1 X[k, :] (columns
//      < end of block k; X starts as I), with L_kk^-1 from step k - 1;
//   -- barrier --
//   2. CTA 0 updates the next diagonal block, A_{k+1,k+1} -= L_{k+1,k}
//      L_{k+1,k}', and factors and inverts it in shared memory (a rank-1
//      update per column; the inverse row by row, eight lanes per column):
//      the diagonal block of step k + 1 is ready when step k ends.  The other
//      CTAs take, round robin, the rest of the trailing lower triangle,
//      A_IJ -= L_Ik L_Jk' (I >= J > k), and the inverse's update
//      X_IJ -= L_Ik X_kJ (I > k, J <= k), 32 x 32 output tiles, loading
//      their next tile's operands into registers while they update the
//      current one;
//   -- barrier --
// FP64 throughout.  A non-positive pivot sets NOT_SPD (info = row_base + row)
// and every CTA leaves at the next barrier.
constexpr int kPotrfThreads = 256;
constexpr int kTileLoads = kBlk * kBlk / kPotrfThreads;  // operand elements per thread and tile

// C (32 x 32, rows r0.., cols c0.. of a column-major matrix) -= A B' or A B:
// a, b are 32 x 32 operand blocks already in shared memory as [row][k].
__device__ __forceinline__ void tile_update32(double *C, int ldc, const double (*a)[kBlk + 1],
                                              const double (*b)[kBlk + 1], int rows, int cols, bool lower_only) {
    const int tid = threadIdx.x, tr = (tid & 15) * 2, tc = (tid >> 4) * 2;
    // the C entries are read before the product, so that their latency
    // overlaps with it (only this CTA updates this tile in this step)
    double cv[2][2];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int r = tr + x, c = tc + y;
            cv[x][y] = (r < rows && c < cols && (!lower_only || c <= r)) ? __ldcg(C + (int64_t)c * ldc + r) : 0.0;
        }
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll 8
    for (int k = 0; k < kBlk; ++k) {
        const double a0 = a[tr][k], a1 = a[tr + 1][k], b0 = b[tc][k], b1 = b[tc + 1][k];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
    }
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int r = tr + x, c = tc + y;
            if (r < rows && c < cols && (!lower_only || c <= r)) C[(int64_t)c * ldc + r] = cv[x][y] - acc[x][y];
        }
}

// The same update in float-float pairs (the inverse X on the paired paths):
// C (pairs) -= A B with a, b pairs in shared memory as [row][k].
__device__ __forceinline__ void tile_update32_ff(float2 *C, int ldc, const float2 (*a)[kBlk + 1],
                                                 const float2 (*b)[kBlk + 1], int rows, int cols) {
    const int tid = threadIdx.x, tr = (tid & 15) * 2, tc = (tid >> 4) * 2;
    float2 cv[2][2];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int r = tr + x, c = tc + y;
            cv[x][y] = (r < rows && c < cols) ? __ldcg(C + (int64_t)c * ldc + r) : make_float2(0.f, 0.f);
        }
    float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
    for (int k = 0; k < kBlk; ++k) {
        const float2 a0 = a[tr][k], a1 = a[tr + 1][k], b0 = b[tc][k], b1 = b[tc + 1][k];
        df_fma(a0.x, a0.y, b0.x, b0.y, h[0][0], l[0][0]);
        df_fma(a0.x, a0.y, b1.x, b1.y, h[0][1], l[0][1]);
        df_fma(a1.x, a1.y, b0.x, b0.y, h[1][0], l[1][0]);
        df_fma(a1.x, a1.y, b1.x, b1.y, h[1][1], l[1][1]);
    }
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int r = tr + x, c = tc + y;
            if (r < rows && c < cols) {
                const FF d = ff_add(FF{cv[x][y].x, cv[x][y].y}, ff_neg(ff_two_sum(h[x][y], l[x][y])));
                C[(int64_t)c * ldc + r] = make_float2(d.h, d.l);
            }
        }
}

__device__ __forceinline__ float2 ff_split(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// 1 / sqrt(d) for d > 0 (normal): the PTX approximation, then two Newton
// steps y <- y (3 - d y^2) / 2, each squaring the relative error (to about
// an ulp).  One thread forms it per column of a diagonal block, where every
// FP64 instruction holds the FP64 pipe for 64 cycles: this takes fewer
// instructions than a square root followed by a quotient per entry.
__device__ __forceinline__ double rsqrt_newton(double d) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    y = y * fma(-0.5 * d * y, y, 1.5);
    return y * fma(-0.5 * d * y, y, 1.5);
}

// Cholesky of the w x w diagonal block at (p, p) of A by the calling CTA,
// with the block's inverse: L_kk into A (lower; upper part of the block 0),
// L_kk^-1 into Li (32 x 32, row major).  Returns the first failing column
// (non-positive pivot) or -1, the same on every thread.
__device__ int potrf_diag_block(double *A, int lda, int p, int w, double *Li, double (*sa)[kBlk + 1],
                                double (*sl)[kBlk + 1], int *s_bad) {
    const int tid = threadIdx.x;
    for (int e = tid; e < kBlk * kBlk; e += kPotrfThreads) {
        const int r = e % kBlk, c = e / kBlk;
        sa[r][c] = (r < w && c < w && c <= r) ? __ldcg(A + (int64_t)(p + c) * lda + p + r) : 0.0;
    }
    if (tid == 0) *s_bad = -1;
    __syncthreads();
    // right-looking Cholesky of the block, one column at a time, the updates
    // spread over the CTA's threads; the pivot's reciprocal is kept in the
    // padding column sa[c][kBlk] (the column is scaled by it, and the
    // inverse below divides by the pivots through it)
    for (int c = 0; c < w; ++c) {
        if (tid == 0) {
            const double d = sa[c][c];
            if (!(d > 0.0)) {
                *s_bad = c;
            } else {
                const double y = rsqrt_newton(d);
                sa[c][c] = d * y;
                sa[c][kBlk] = y;
            }
        }
        __syncthreads();
        if (*s_bad >= 0) break;  // read after the barrier: uniform
        const double rpiv = sa[c][kBlk];
        for (int r = c + 1 + tid; r < w; r += kPotrfThreads) sa[r][c] *= rpiv;
        __syncthreads();
        const int nr = w - c - 1;
        for (int e = tid; e < nr * nr; e += kPotrfThreads) {
            const int r = c + 1 + e % nr, cc = c + 1 + e / nr;
            if (cc <= r) sa[r][cc] -= sa[r][c] * sa[cc][c];
        }
        __syncthreads();
    }
    const int bad = *s_bad;
    if (bad >= 0) return bad;
    // inverse of the lower triangular block, row by row: column c by the 8
    // lanes 8c .. 8c+7 (one warp holds four columns), each summing every 8th
    // term, then a shuffle reduction
    const int c = tid >> 3, q = tid & 7;
    for (int r = 0; r < kBlk; ++r) {
        double part = 0.0;
        if (c < w && r < w && r > c)
            for (int k = c + q; k < r; k += 8) part = fma(sa[r][k], sl[k][c], part);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 4);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 2);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 1);
        if (q == 0) {
            double v = 0.0;
            if (c < w && r < w && r >= c) v = ((r == c ? 1.0 : 0.0) - part) * sa[r][kBlk];
            sl[r][c] = v;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int e = tid; e < kBlk * kBlk; e += kPotrfThreads) {
        const int r = e % kBlk, cc = e / kBlk;
        if (r < w && cc < w) A[(int64_t)(p + cc) * lda + p + r] = (cc <= r) ? sa[r][cc] : 0.0;
        Li[r * kBlk + cc] = sl[r][cc];
    }
    return -1;
}

// `scratch`: 32 x 1024 doubles for the diagonal block inverses, then one
// word through which CTA 0 tells the cluster to stop (the context's status
// word may be set by kernels on other streams at any time, so the CTAs do not
// each read it to decide).
// One cluster per job (blockIdx.x / kCl): the diagonal tiles of several
// factorisations in one launch (the jobs travel in the kernel parameters).
// kFF: the inverse X in float-float pairs on the FP32 pipe (stored as pairs
// in X's memory while the kernel runs, as doubles hi + lo at the end); the
// Cholesky factor stays FP64.  The paired paths use X only in products they
// run in paired FP32.
template <int kCl, bool kFF>
__global__ void __launch_bounds__(kPotrfThreads) k_potrf_inv(const PotrfBatch jobs) {
    const PotrfJob J = jobs.job[blockIdx.x / kCl];
    double *const A = J.A, *const X = J.X, *const scratch = J.scratch;
    const int lda = J.lda, m = J.m, ldx = J.ldx;
    DevStatus *const st = J.st;
    const long long row_base = J.row_base;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), tid = threadIdx.x;
    const int gtid = rank * kPotrfThreads + tid, gthreads = kCl * kPotrfThreads;
    __shared__ double sa[kBlk][kBlk + 1], sb[kBlk][kBlk + 1], sl[kBlk][kBlk + 1];
    __shared__ float2 slf[kFF ? kBlk : 1][kBlk + 1];  // L_kk^-1 as pairs (kFF)
    __shared__ int s_bad;
    float2 *const X2 = reinterpret_cast<float2 *>(X);
    float2 (*const saf)[kBlk + 1] = reinterpret_cast<float2 (*)[kBlk + 1]>(sa);
    float2 (*const sbf)[kBlk + 1] = reinterpret_cast<float2 (*)[kBlk + 1]>(sb);
    const int nbk = (m + kBlk - 1) / kBlk;
    double *dinv = scratch;
    long long *stop = reinterpret_cast<long long *>(scratch + (int64_t)kBlk * kBlk * kBlk);
    // X = I; CTA 0 factors the first diagonal block
    for (int64_t e = gtid; e < (int64_t)m * m; e += gthreads) {
        const int r = (int)(e % m), c = (int)(e / m);
        if constexpr (kFF) X2[(int64_t)c * ldx + r] = make_float2(r == c ? 1.f : 0.f, 0.f);
        else X[(int64_t)c * ldx + r] = (r == c) ? 1.0 : 0.0;
    }
    if (rank == 0) {
        // one read of the status word decides for the whole CTA (another
        // stream's kernel may set it at any time)
        if (tid == 0) s_bad = __ldcg(&st->code) ? 1 : 0;
        __syncthreads();
        long long halt = s_bad ? 1LL : 0LL;
        __syncthreads();
        if (!halt) {
            const int bad = potrf_diag_block(A, lda, 0, min(kBlk, m), dinv, sa, sl, &s_bad);
            if (bad >= 0) {
                if (tid == 0) set_status(st, TLR_ERR_NOT_SPD, row_base + bad);
                halt = 1;
            }
        }
        if (tid == 0) __stcg(stop, halt);
    }
    cl.sync();
    if (__ldcg(stop)) return;
    for (int kb = 0; kb < nbk; ++kb) {
        const int p = kb * kBlk, w = min(kBlk, m - p);
        const double *Li = dinv + (int64_t)kb * kBlk * kBlk;  // L_kk^-1, row major
        // 1. panel rows below the block: x <- a L_kk^-T, x_c = sum_{k<=c} a_k Linv[c][k];
        //    inverse block row: X[k-block, c] <- L_kk^-1 X[k-block, c], c < p + w
        for (int e = tid; e < kBlk * kBlk; e += kPotrfThreads) {
            const double v = __ldcg(Li + e);
            sl[e / kBlk][e % kBlk] = v;
            if constexpr (kFF) slf[e / kBlk][e % kBlk] = ff_split(v);
        }
        __syncthreads();
        // rows and columns dealt to the CTAs in turn (gq = tid * kCl + rank), so
        // that every CTA's FP64 pipe takes a share (a 32-term chain each)
        const int gq = tid * kCl + rank;
        for (int r = p + w + gq; r < m; r += gthreads) {
            double a[kBlk];
#pragma unroll
            for (int k = 0; k < kBlk; ++k) a[k] = k < w ? __ldcg(A + (int64_t)(p + k) * lda + r) : 0.0;
#pragma unroll
            for (int c = 0; c < kBlk; ++c) {
                if (c >= w) break;
                double x = 0.0;
#pragma unroll
                for (int k = 0; k <= c; ++k) x = fma(a[k], sl[c][k], x);
                A[(int64_t)(p + c) * lda + r] = x;
            }
        }
        for (int c = gq; c < p + w; c += gthreads) {
            if constexpr (kFF) {
                float2 x[kBlk];
#pragma unroll
                for (int k = 0; k < kBlk; ++k)
                    x[k] = k < w ? __ldcg(X2 + (int64_t)c * ldx + p + k) : make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < kBlk; ++r) {
                    if (r >= w) break;
                    float vh = 0.f, vl = 0.f;
#pragma unroll
                    for (int k = 0; k <= r; ++k) df_fma(slf[r][k].x, slf[r][k].y, x[k].x, x[k].y, vh, vl);
                    const FF v = ff_two_sum(vh, vl);
                    X2[(int64_t)c * ldx + p + r] = make_float2(v.h, v.l);
                }
            } else {
                double x[kBlk];
#pragma unroll
                for (int k = 0; k < kBlk; ++k) x[k] = k < w ? __ldcg(X + (int64_t)c * ldx + p + k) : 0.0;
#pragma unroll
                for (int r = 0; r < kBlk; ++r) {
                    if (r >= w) break;
                    double v = 0.0;
#pragma unroll
                    for (int k = 0; k <= r; ++k) v = fma(sl[r][k], x[k], v);
                    X[(int64_t)c * ldx + p + r] = v;
                }
            }
        }
        cl.sync();
        if (kb + 1 >= nbk) break;
        // 2. trailing and inverse updates by this block column; CTA 0 also
        //    prepares the next diagonal block
        const int nt = nbk - kb - 1;            // block rows below
        const int ntr = nt * (nt + 1) / 2;      // trailing tiles (I >= J > kb); tile 0 is (kb+1, kb+1)
        const int ntot = ntr + nt * (kb + 1);   // + inverse tiles (I > kb, J <= kb)
        // tile t -> operands: trailing (I, J): C = A_IJ, a = L_I,kb, b = L_J,kb (as [row][k]);
        //                     inverse (I, J): C = X_IJ, a = L_I,kb, b = X_kb,J (as [col][k])
        auto tile_of = [&](int t, bool &inv, int &I, int &Jb) {
            if (t < ntr) {
                int bi = 0, rem = t;
                while (rem > bi) { rem -= bi + 1; ++bi; }
                inv = false;
                I = kb + 1 + bi;
                Jb = kb + 1 + rem;
            } else {
                const int u = t - ntr;
                inv = true;
                I = kb + 1 + u % nt;
                Jb = u / nt;
            }
        };
        double ra[kTileLoads], rb[kTileLoads];
        float2 rbf[kTileLoads];
        auto fetch = [&](int t) {
            bool inv;
            int I, Jb;
            tile_of(t, inv, I, Jb);
            const int ri = I * kBlk, cj = Jb * kBlk, rows = min(kBlk, m - ri), cols = min(kBlk, m - cj);
#pragma unroll
            for (int u = 0; u < kTileLoads; ++u) {
                const int e = tid + u * kPotrfThreads, r = e % kBlk, k = e / kBlk;
                ra[u] = (r < rows && k < w) ? __ldcg(A + (int64_t)(p + k) * lda + ri + r) : 0.0;
                if (kFF && inv)
                    rbf[u] = (r < cols && k < w) ? __ldcg(X2 + (int64_t)(cj + r) * ldx + p + k) : make_float2(0.f, 0.f);
                else if (inv) rb[u] = (r < cols && k < w) ? __ldcg(X + (int64_t)(cj + r) * ldx + p + k) : 0.0;
                else rb[u] = (r < cols && k < w) ? __ldcg(A + (int64_t)(p + k) * lda + cj + r) : 0.0;
            }
        };
        auto apply = [&](int t) {
            bool inv;
            int I, Jb;
            tile_of(t, inv, I, Jb);
            const int ri = I * kBlk, cj = Jb * kBlk, rows = min(kBlk, m - ri), cols = min(kBlk, m - cj);
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kTileLoads; ++u) {
                const int e = tid + u * kPotrfThreads;
                if (kFF && inv) {
                    saf[e % kBlk][e / kBlk] = ff_split(ra[u]);
                    sbf[e % kBlk][e / kBlk] = rbf[u];
                } else {
                    sa[e % kBlk][e / kBlk] = ra[u];
                    sb[e % kBlk][e / kBlk] = rb[u];
                }
            }
            __syncthreads();
            return inv ? (X + (int64_t)cj * ldx + ri) : (A + (int64_t)cj * lda + ri);
        };
        if (rank == 0) {
            // tile (kb+1, kb+1), then the next diagonal block
            fetch(0);
            double *C = apply(0);
            tile_update32(C, lda, sa, sb, min(kBlk, m - (kb + 1) * kBlk), min(kBlk, m - (kb + 1) * kBlk), true);
            __syncthreads();
            const int pn = (kb + 1) * kBlk, wn = min(kBlk, m - pn);
            const int bad = potrf_diag_block(A, lda, pn, wn, dinv + (int64_t)(kb + 1) * kBlk * kBlk, sa, sl, &s_bad);
            if (bad >= 0 && tid == 0) {
                set_status(st, TLR_ERR_NOT_SPD, row_base + pn + bad);
                __stcg(stop, 1LL);
            }
        } else {
            const int step = kCl - 1;
            if (1 + rank - 1 < ntot) fetch(1 + rank - 1);
            for (int t = 1 + rank - 1; t < ntot; t += step) {
                bool inv;
                int I, Jb;
                tile_of(t, inv, I, Jb);
                const int ri = I * kBlk, cj = Jb * kBlk, rows = min(kBlk, m - ri), cols = min(kBlk, m - cj);
                double *C = apply(t);
                if (t + step < ntot) fetch(t + step);
                if (kFF && inv) tile_update32_ff(reinterpret_cast<float2 *>(C), ldx, saf, sbf, rows, cols);
                else tile_update32(C, inv ? ldx : lda, sa, sb, rows, cols, !inv && I == Jb);
            }
        }
        cl.sync();
        if (__ldcg(stop)) return;  // written by CTA 0 only, before the barrier
    }
    // zero the strict upper triangle of the factor; the paired inverse to doubles
    for (int64_t e = gtid; e < (int64_t)m * m; e += gthreads) {
        const int r = (int)(e % m), c = (int)(e / m);
        if (r < c) A[(int64_t)c * lda + r] = 0.0;
        if constexpr (kFF) {
            const float2 v = X2[(int64_t)c * ldx + r];
            X[(int64_t)c * ldx + r] = (double)v.x + (double)v.y;
        }
    }
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

void potrf_inv_batched(tlr_ctx *ctx, cudaStream_t s, std::vector<PotrfJob> jobs, bool ff_inverse) {
    std::vector<PotrfJob> act;
    for (const PotrfJob &J : jobs) {
        if (J.m <= 0) continue;
        if (J.m > kBlk * kBlk) throw make_error(TLR_ERR_ARG, "tile too large for the cluster POTRF (%d)", J.m);
        act.push_back(J);
    }
    if (act.empty()) return;
    if ((int)act.size() > kMaxGroup) throw make_error(TLR_ERR_ARG, "more than %d diagonal tiles in one launch", kMaxGroup);
    // scratch per job: the diagonal-block inverses and the cluster's stop word
    const size_t per = (size_t)kBlk * kBlk * kBlk + 8;
    if ((int)act.size() > ctx->potrf_scratch_jobs) {
        if (ctx->d_potrf_scratch) TLR_CUDA_TRY(cudaFree(ctx->d_potrf_scratch));  // syncs the device
        ctx->d_potrf_scratch = nullptr;
        ctx->potrf_scratch_jobs = 0;
        const int want = std::max((int)act.size(), 2 * ctx->potrf_scratch_jobs);
        TLR_CUDA_TRY(cudaMalloc(&ctx->d_potrf_scratch, per * want * sizeof(double)));
        ctx->potrf_scratch_jobs = want;
    }
    PotrfBatch b{};
    for (size_t q = 0; q < act.size(); ++q) {
        b.job[q] = act[q];
        b.job[q].scratch = ctx->d_potrf_scratch + per * q;
    }
    static std::once_flag once;
    static int csize = 8;  // 16 CTAs where the device runs such clusters, else 8
    std::call_once(once, [] {
        if (cudaFuncSetAttribute(k_potrf_inv<16, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_potrf_inv<16, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(kPotrfThreads);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 16;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_potrf_inv<16, true>, &cfg) == cudaSuccess && nclusters > 0)
                csize = 16;
        }
        cudaGetLastError();  // clear any error of the queries
    });
    const int nc = (int)act.size();
    if (csize == 16) {
        if (ff_inverse) launch_clustered(k_potrf_inv<16, true>, 16, nc, kPotrfThreads, 0, s, b);
        else launch_clustered(k_potrf_inv<16, false>, 16, nc, kPotrfThreads, 0, s, b);
    } else {
        if (ff_inverse) launch_clustered(k_potrf_inv<8, true>, 8, nc, kPotrfThreads, 0, s, b);
        else launch_clustered(k_potrf_inv<8, false>, 8, nc, kPotrfThreads, 0, s, b);
    }
}

void potrf_inv(tlr_ctx *ctx, cudaStream_t s, double *A, int lda, int m, double *X, int ldx, long long row_base) {
    potrf_inv_batched(ctx, s, {PotrfJob{A, lda, m, X, ldx, nullptr, ctx->d_status, row_base}});
}

// acc[0] += sum_r log A[r, r]  (one block, fixed reduction order); if maxinv
// is not null, *maxinv = max(*maxinv, max_r 1 / A[r, r]^2) (the largest
// inverse squared pivot, i.e. the smallest conditional variance seen so far;
// positive doubles order like their bit patterns, so an integer atomicMax
// keeps the result independent of launch order).
__global__ void k_diag_logsum(const double *__restrict__ A, int lda, int m, double *acc,
                              const DevStatus *st, double *maxinv) {
    __shared__ double part[256], pmax[256];
    double s = 0.0, mx = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const double d = A[(int64_t)r * lda + r];
        s += log(d);
        mx = fmax(mx, 1.0 / (d * d));
    }
    part[threadIdx.x] = s;
    pmax[threadIdx.x] = mx;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            part[threadIdx.x] += part[threadIdx.x + h];
            pmax[threadIdx.x] = fmax(pmax[threadIdx.x], pmax[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && !st->code) {
        acc[0] += part[0];
        if (maxinv && pmax[0] > 0.0 && pmax[0] <= 1.7e308)
            atomicMax(reinterpret_cast<unsigned long long *>(maxinv), (unsigned long long)__double_as_longlong(pmax[0]));
    }
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

void diag_logsum(cudaStream_t s, const double *A, int lda, int m, double *acc, const DevStatus *st, double *maxinv) {
    launch(k_diag_logsum, 1, 256, 0, s, A, lda, m, acc, st, maxinv);
    TLR_CHECK_LAUNCH();
}

void sumsq(cudaStream_t s, const double *v, int m, double *acc) {
    launch(k_sumsq, 1, 256, 0, s, v, m, acc);
    TLR_CHECK_LAUNCH();
}

}  // namespace tlr

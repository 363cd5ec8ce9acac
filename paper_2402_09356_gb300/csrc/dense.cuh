// Dense FP64 tile operations (declarations; see dense.cu).
#pragma once

#include "common.cuh"

namespace tlr {

// One right-hand side matrix of a batched triangular solve: m x ncols, column
// major with leading dimension ld, solved in place.
struct RhsDesc {
    double *B;
    int ncols;
    int ld;
};

// A = L L' in place (lower; strict upper zeroed) and X = L^-1 (m x m, lower,
// ld ldx) in one launch on one thread-block cluster; m <= 1024.  A
// non-positive pivot sets NOT_SPD (info = row_base + local row); X is then
// not written.
void potrf_inv(tlr_ctx *ctx, cudaStream_t s, double *A, int lda, int m, double *X, int ldx, long long row_base);

// The same for several tiles in one launch (one cluster each); every job
// reports a non-positive pivot in its own status word st.  scratch is set by
// the call.
struct PotrfJob {
    double *A;
    int lda, m;
    double *X;
    int ldx;
    double *scratch;
    DevStatus *st;
    long long row_base;
};
struct PotrfBatch {
    PotrfJob job[kMaxGroup];
};
// ff_inverse: X in float-float arithmetic (~1e-14 relative), the factor in
// FP64 (the paired-FP32 paths, whose products with X are paired FP32).
void potrf_inv_batched(tlr_ctx *ctx, cudaStream_t s, std::vector<PotrfJob> jobs, bool ff_inverse = false);

// B <- L^-1 B for every right-hand side matrix (L lower triangular m x m).
void trsm_left_lower(tlr_ctx *ctx, cudaStream_t s, const double *L, int ldl, int m,
                     const std::vector<RhsDesc> &rhs);

// acc[0] += sum_r log A[r, r] (skipped once the status word holds an error);
// maxinv (optional): running maximum of 1 / A[r, r]^2.
void diag_logsum(cudaStream_t s, const double *A, int lda, int m, double *acc, const DevStatus *st,
                 double *maxinv = nullptr);

// acc[0] += |v|^2
void sumsq(cudaStream_t s, const double *v, int m, double *acc);

}  // namespace tlr

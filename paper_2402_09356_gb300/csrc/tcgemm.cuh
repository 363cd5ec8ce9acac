// Tensor-core products for the mixed-precision path (declarations; see tcgemm.cu).
//
// C = alpha op(A) op(B) (+ the linear or Matern epilogue) for FP64 operands on
// the 5th-generation tensor cores (tcgen05), by splitting every operand into
// S BF16 slices with a power-of-two scale per row and 64-wide chunk of the
// inner dimension (the error-free splitting of Ozaki, Ogita and Oishi,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 2012):
//   x = 2^e (c_0 2^-8 + c_1 2^-16 + ... + c_{S-1} 2^-8S) + O(2^(e-8S)),
// c_p integers of at most 8 significant bits, so every slice is an exact
// BF16 number and every slice product is exact in FP32.  The products of
// slice pairs (p, q) with p + q <= S - 1 are accumulated in TMEM per order
// p + q (orders 0, 1 and 2 exactly: within a 64-wide chunk their sums stay
// below 2^24 units; orders >= 3, weighted 2^-24 and below, share one
// accumulator) and added, chunk by chunk, into float-float accumulators
// (Dekker 1971) with the chunk's scales.  With S = 5 a product carries about
// 40 significant bits relative to the scale of its row and column: the
// rounding noise of a panel update stays ~1e-12, below the compression
// thresholds of the workloads (eps >= 1e-9).  S = 1 is the plain BF16
// product with FP32 accumulation and per-chunk scaling.
#pragma once

#include "common.cuh"
#include "gemm.cuh"
#include "matern.cuh"

namespace tlr {

constexpr int kTcSlicesDefault = 5;

// Whether the tensor-core products can run on the current device (sm_103a
// kernels loaded, enough opt-in shared memory).  Thread safe, cached.
bool tc_available();

// C_b = alpha op(A_b) op(B_b) + beta C_b for every problem (A, B, C, m, n, k,
// lda, ldb, ldc of GemmProb; A2/B2 unused).  slices: 1 or 5.  Operands that
// appear in several problems (same pointer, leading dimension, transposition
// and size) are split once.
// light: two pipeline stages instead of three (100 KB of shared memory per
// CTA instead of 150 KB), for products running beside critical-path work.
void gemm_tc(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs, double alpha,
             double beta, int slices = kTcSlicesDefault, bool light = false);

// The panel update with the Matern epilogue (B transposed): C = Sigma + alpha A B'.
// ctas_per_sm > 0 keeps the product to one CTA per SM with two pipeline
// stages (room for the critical-path kernels beside it).
void gemm_tc_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs, double alpha,
                    const double *xy, int64_t n, const MaternParams &P, int slices = kTcSlicesDefault,
                    int ctas_per_sm = 0);

// Test hook (C ABI tlr_gemm_tc): one product C = alpha op(A) op(B) + beta C.
void gemm_tc_single(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                    const double *A, int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices);

}  // namespace tlr

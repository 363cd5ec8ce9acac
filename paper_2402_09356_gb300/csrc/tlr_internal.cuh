// Internal interfaces between the TLR factorisation (tlr.cu), the pool (pool.cu) and the C ABI (api.cu).
#pragma once

#include <functional>
#include <string>

#include "common.cuh"
#include "matern.cuh"

namespace tlr {

// A batched matrix copy: dst (m x n, ld ldd) = src (ld lds), or 0 if src is null.
struct CopyDesc {
    const double *src;
    int lds;
    double *dst;
    int ldd;
    int m, n;
};

void copy_batched(tlr_ctx *ctx, cudaStream_t s, const std::vector<CopyDesc> &descs);

constexpr int kStages = 5;

// finer profiling buckets of the factorisation (device ms, summed over columns)
enum DetailBucket {
    kDetBuild,       // P_j, Q_j operands of a main-stream panel update
    kDetCorrect,     // look-ahead: correction of the panel by the previous column
    kDetAheadWait,   // main stream waiting for the look-ahead stream
    kDetSolveUpd,    // fused forward-solve update of y_j
    kDetSplit,       // paired-FP32 copy of the panel for the compression
    kDetPanel,       // panel update GEMM on the main stream
    kDetDiagCopy,    // diagonal tile copy and fork to the side stream
    kDetCompress,    // off-diagonal compression
    kDetJoin,        // waiting for the side stream (POTRF + inverse)
    kDetTrsm,        // V_ij <- L_jj^-1 V_ij
    kDetSolve,       // y_j <- L_jj^-1 y_j, log-determinant and |y|^2 terms, V_j' y_j
    kDetGram,        // G_j = V_j' V_j
    kDetPotrf,       // side stream: dense POTRF of the diagonal tile and L_jj^-1 (one launch)
    kDetInverse,     // unused (the inverse is part of the POTRF launch)
    kDetAheadBuild,  // look-ahead stream: P, Q operands of the next column's update
    kDetAheadPanel,  // look-ahead stream: the next column's panel GEMM (Matern epilogue)
    kDetail
};

enum class FactorMode {
    Matern,  // tiles generated from the Matern kernel inside the panel update (likelihood path)
    Tlr      // tiles taken from the compressed input held in the matrix (tlr_potrf)
};

struct FactorStats {
    double flops = 0.0;           // floating-point operations counted from the rank map
    double gemm_flops = 0.0;      // of which: panel update GEMMs
    double matern_entries = 0.0;  // covariance entries evaluated in the panel epilogues
    int panel_launches = 0;
    float gemm_ms = 0.f;          // device time of the panel GEMMs (when ctx->profile)
    // device time per stage (when ctx->profile): low-rank operand build, panel
    // update GEMM, diagonal POTRF, compression, TRSM of V
    float stage_ms[kStages] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float detail_ms[kDetail] = {};
};

void profile_events(tlr_ctx *ctx, int count);
void upload_ranks(tlr_mat *M, cudaStream_t s);
// TLR Cholesky.  With z, y and acc given, the forward solve of Eq. 1.2 is fused
// in: y = L^-1 z (z, y device, ordered; may alias), acc[0] += sum log L_ii,
// acc[1] += |y|^2, acc[2] = max(acc[2], max_i 1 / L_ii^2).  With df (Matern mode only), the panel update and the
// compression's sampling and projection products run in paired-FP32
// arithmetic; everything else stays FP64.  With tc as well, those products,
// the correction by the previous column, V <- L^-1 V and the Gram matrices
// run on the tensor cores (BF16 slices, tcgemm.cuh); the compression's QR
// stays paired FP32.
void factor(tlr_ctx *ctx, cudaStream_t s, tlr_mat *M, FactorMode mode, const double *xy,
            const MaternParams *P, double tau, FactorStats *stats, long long *info,
            const double *z = nullptr, double *y = nullptr, double *acc = nullptr, bool df = false,
            bool tc = false);

// One factorisation of a group advanced together by factor_group.
struct FactorItem {
    tlr_mat *M = nullptr;
    const double *xy = nullptr;       // Matern mode: ordered locations (device, SoA)
    const MaternParams *P = nullptr;  // Matern mode: parameters with their table built
    double tau = 0.0;                 // absolute compression accuracy
    FactorStats *stats = nullptr;     // the first item's also receives the call's profiling times
    long long *info = nullptr;
    const double *z = nullptr;        // fused solve (optional), as for factor
    double *y = nullptr;
    double *acc = nullptr;
    int err = TLR_OK;                 // output: the status that stopped this factorisation
    std::string msg;
};

// The factorisations of `items` (at most kMaxGroup; one only in Tlr mode)
// column by column in lockstep on one context: every step of column j is one
// launch for all of them (panel products and generation, diagonal POTRF
// clusters, every compression launch class, V <- L^-1 V, Gram matrices), so
// the uneven-rank tiles of several factorisations share each launch.  Each
// factorisation computes exactly what factor would compute for it alone.
// A factorisation that meets a non-positive pivot, a non-finite tile or a
// rank that does not fit stops with err / msg / *info set; the others go on.
// Status words: with one item the context's word; with G > 1 items, word
// 1 + g of ctx->d_status for item g (the caller resets words 0..G), word 0
// for device-wide failures, which stop the call with an exception.
void factor_group(tlr_ctx *ctx, cudaStream_t s, std::vector<FactorItem> &items, FactorMode mode, bool df,
                  bool tc);
void forward_solve(tlr_ctx *ctx, cudaStream_t s, const tlr_mat *M, const double *z, double *y,
                   double *acc);
void lmul(tlr_ctx *ctx, cudaStream_t s, const tlr_mat *M, const double *w, double *z);
void compress_packed(tlr_ctx *ctx, cudaStream_t s, const double *tiles, tlr_mat *M, double tau,
                     long long *info);

// ordering (order.cu)
void order_sfc(const double *xy, int64_t n, int method, uint64_t seed, int64_t *perm, uint32_t *codes,
               cudaStream_t s);
void order_kdtree(const double *xy, int64_t n, int64_t *perm, cudaStream_t s);
void order_maxmin(const double *xy, int64_t n, int64_t *perm, cudaStream_t s, int num_sms);
void order_identity(int64_t n, int64_t *perm, cudaStream_t s);
void permute_xy(const double *xy, const int64_t *perm, int64_t n, int quantize, double *out, cudaStream_t s);
void gather(const int64_t *perm, const double *src, int64_t n, double *dst, cudaStream_t s);

// covariance (matern.cu)
void generate_tiles(const double *xy, int64_t n, int nb, const MaternParams &P, double *tiles, cudaStream_t s);
void matern_vec(const double *d, int64_t m, const MaternParams &P, double *out, cudaStream_t s);
// T[c * ld + r] = C(s_{ri0 + r}, s_{ci0 + c}) for r < rows, c < cols (0 past n).
void generate_panel(const double *xy, int64_t n, int64_t ri0, int64_t ci0, int rows, int cols,
                    const MaternParams &P, double *T, int ld, cudaStream_t s);

// One entry of a batched evaluation (tlr_loglik_batch): inputs, then the
// entry's own status and message (NOT_SPD, RANK, NAN) on return.
struct BatchEntry {
    const double *xy = nullptr, *z = nullptr;
    int64_t n = 0;
    tlr_theta theta{};
    const tlr_opts *opts = nullptr;
    tlr_mat *L = nullptr;
    tlr_result *out = nullptr;
    int status = TLR_OK;
    std::string msg;
};
// tlr_loglik_batch on entries (validated here); errors of the whole call throw.
void loglik_batch(tlr_ctx *ctx, std::vector<BatchEntry> &es, cudaStream_t s);

// Bounds of a maximum-likelihood search: positive, finite, lo <= hi.
bool mle_bounds_ok(tlr_theta lo, tlr_theta hi);

// Derivative-free maximum-likelihood search (Sec. 5.1): Nelder-Mead in
// log(theta) over the box [lo, hi] (bounds by clamping) on negll(theta) =
// -l(theta), +inf for a failed evaluation.  Stops when the simplex spread in
// -l falls below tol * (1 + |l|), its size in log(theta) below 1e-8, or after
// max_iter evaluations.  Throws NOT_SPD if no evaluation was finite.
void mle_nelder_mead(const std::function<double(tlr_theta)> &negll, tlr_theta theta0, tlr_theta lo,
                     tlr_theta hi, double tol, int max_iter, tlr_theta *theta_hat, double *ll_hat, int *iters);

// Compact slot layout of a TLR matrix from a rank map (host, NT x NT, r_ij at
// i * NT + j for i > j; empty = no map): each off-diagonal tile gets
// cap = min(maxrank, r + max(8, r / 4) rounded up to 8) columns, and an
// overflow arena of max(sum cap / 8, 4 maxrank) columns follows.  Fills the
// layout fields of M (base_off, cap, arena) and returns the total number of
// columns U and V need; with no map, the uniform layout (noff * maxrank).
int64_t plan_slots(tlr_mat *M, const std::vector<int32_t> &hint);

}  // namespace tlr

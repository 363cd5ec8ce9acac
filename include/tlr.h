/*
 * tlr.h -- C ABI of the GB300 (sm_103a) Tile Low-Rank Matern log-likelihood.
 *
 * The library evaluates the Gaussian log-likelihood of Eq. 1.2,
 *     l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 Z' Sigma(theta)^-1 Z,
 * for the Matern covariance of Eq. 4.2 (theta = sigma2, beta, nu), under the
 * Tile Low-Rank (TLR) approximation of Sec. 2 and after one of the spatial
 * orderings of Sec. 3.  Every step runs in CUDA kernels of this library.
 *
 * Conventions shared by every call
 *  - Return value: TLR_OK (0) or one TLR_ERR_* code.  A failing call leaves a
 *    message in tlr_last_error(ctx).  No C++ exception crosses this boundary.
 *  - "device" pointers are CUDA global-memory pointers of the context's
 *    device; "host" pointers are ordinary CPU memory.  The caller owns every
 *    pointer it passes; the library keeps none of them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream ordered; a call syncs the stream only where it
 *    returns a value on the host (documented per call).
 *  - Locations are SoA float64: xy[0..n) = x, xy[n..2n) = y.
 *  - Matrix tiles are column major.  The tile size is nb; NT = ceil(n / nb);
 *    tile t covers rows [t nb, min(n, (t+1) nb)) and has m_t rows.
 *  - A context is used by one host thread at a time (a pool, below, by any).
 */
#ifndef TLR_H
#define TLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define TLR_OK            0
#define TLR_ERR_ARG       1  /* invalid argument (sizes, pointers, theta, flags) */
#define TLR_ERR_CUDA      2  /* a CUDA runtime call failed */
#define TLR_ERR_OOM       3  /* device memory could not be allocated */
#define TLR_ERR_RANK      4  /* an off-diagonal tile needs rank > maxrank (Sec. 5.2, Table 1 "NA") */
#define TLR_ERR_NOT_SPD   5  /* non-positive pivot in a Cholesky factorisation */
#define TLR_ERR_TIMEOUT   6  /* a bounded device wait gave up */
#define TLR_ERR_NAN       7  /* a non-finite value was produced */

/* ---- orderings (Sec. 3) --------------------------------------------------- */
#define TLR_ORDER_IDENTITY 0 /* generation order: the paper's "no order" (Sec. 5.1) */
#define TLR_ORDER_RANDOM   1 /* stable sort of splitmix64(seed ^ i) >> 32 */
#define TLR_ORDER_MORTON   2 /* Sec. 3.1.1: interleaved bits of 16-bit coordinates */
#define TLR_ORDER_HILBERT  3 /* Sec. 3.1.2: Hilbert index, orientation of Figure 3 */
#define TLR_ORDER_KDTREE   4 /* Sec. 3.2: median splits on the widest dimension, in-order */
#define TLR_ORDER_MAXMIN   5 /* Sec. 3.3.1 (Guinness 2018): maximum-minimum distance */

/* tlr_order flags */
#define TLR_ORDER_QUANTIZE 1u /* xy_out holds decoded coordinates q / 65535 (Sec. 3.1, "Decoding") */

/* precision of the off-diagonal products (tlr_opts.precision) */
#define TLR_PREC_FP64 0  /* every operation in FP64 */
/* Mixed: the dense products of the off-diagonal work -- the panel update
 * T_ij = A_ij - sum_k L_ik L_jk' and the compression's sampling T Omega and
 * projection T' Q -- run in paired-FP32 arithmetic on the FP32 pipe (each
 * operand split into two FP32 words, products and sums carried to about 46
 * significant bits); storage, the Matern evaluation, QR/SVD, the diagonal
 * POTRF, the log-determinant and the solve stay FP64. */
#define TLR_PREC_MIXED 1
/* Auto: paired-FP32 rounding (about 1e-14 relative per product) is amplified
 * by the covariance's conditioning, so the mixed path is used only where the
 * factor shows a well-conditioned covariance: smallest squared pivot
 * min_i L_ii^2 (the smallest conditional variance of a location given the
 * ones before it) at least TLR_AUTO_PIVOT2 sigma2.  A matrix whose previous
 * likelihood fell below goes to the FP64 path at once; otherwise the mixed
 * path runs, and where its factor falls below (or meets a non-positive
 * pivot) the FP64 path runs again from the same starting rank map and its
 * result is returned.  tlr_result.precision_used says which.  The threshold
 * comes from a measurement: over 444 batched evaluations (256 datasets, n
 * 2k-20k, nu up to 2.5, data drawn from each dataset's model Z = L w, each
 * path from its own rank-map history) every mixed result whose factor stayed
 * at or above 1e-5 sigma2 was within 6.1e-9 |l| of the FP64 one (8.4e-7 at or
 * above 1e-6), and up to 1.9e-4 below it; 3e-5 keeps a margin. */
#define TLR_PREC_AUTO 2
#define TLR_AUTO_PIVOT2 3e-5
/* Tensor: the mixed path with its dense off-diagonal products -- the panel
 * update (with the Matern epilogue), the correction by the previous column,
 * the compression's sampling and projection, V <- L^-1 V and the Gram
 * matrices V'V -- on the tensor cores (tcgen05): each FP64 operand split into
 * five BF16 slices with a power-of-two scale per row and 64-wide chunk of the
 * inner dimension, slice products accumulated in FP32 in tensor memory and
 * summed in float-float, about 40 significant bits per product (tlr_gemm_tc).
 * The compression's QR runs in paired FP32; storage, the Matern evaluation,
 * the SVD, the diagonal POTRF, the log-determinant and the solve stay FP64.
 * Needs an sm_103a device (TLR_ERR_CUDA otherwise). */
#define TLR_PREC_TENSOR 3

typedef struct tlr_ctx tlr_ctx; /* device, workspace pool, last error, timers */
typedef struct tlr_mat tlr_mat; /* a TLR matrix or TLR Cholesky factor on the device */

typedef struct {
    double sigma2; /* variance, > 0 */
    double beta;   /* range, > 0 */
    double nu;     /* smoothness, > 0 */
} tlr_theta;

typedef struct {
    int32_t nb;        /* tile size, 16 <= nb <= 1024 */
    int32_t maxrank;   /* largest off-diagonal rank stored; <= 0 selects nb / 2 (Sec. 3) */
    double eps;        /* TLR accuracy: singular values <= eps * sigma2 are dropped */
    int32_t precision; /* TLR_PREC_* */
    uint32_t flags;    /* reserved, 0 */
} tlr_opts;

typedef struct {
    double loglik;        /* Eq. 1.2 */
    double logdet;        /* log|Sigma| = 2 sum log L_ii */
    double quad;          /* Z' Sigma^-1 Z = |L^-1 Z|^2 */
    int64_t info;         /* NOT_SPD: global row of the failing pivot; RANK: tile i*NT+j; else -1 */
    int32_t max_rank;     /* largest off-diagonal rank of the factor */
    double mean_rank;     /* mean off-diagonal rank of the factor */
    int64_t offdiag_bytes;/* Table 1 accounting: sum over i>j of (m_i + m_j) r_ij * 8 */
    int64_t dense_bytes;  /* Table 1 "Dense": lower off-diagonal tiles * nb^2 * 8 */
    double flops;         /* floating-point operations counted from the rank map */
    float ms_total;       /* device time of the call (CUDA events on `stream`) */
    int32_t precision_used; /* TLR_PREC_FP64, TLR_PREC_MIXED or TLR_PREC_TENSOR: the path the result comes from */
    double min_pivot2;    /* min_i L_ii^2 over the factor's diagonal (a conditional variance) */
} tlr_result;

/* ---- context -------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Workspaces are taken from the device's default stream-ordered memory pool;
 * the call sets that pool's release threshold to unlimited (for this
 * process), so that freed workspace memory stays cached between tile columns.
 * Errors: TLR_ERR_ARG (out NULL), TLR_ERR_CUDA (no such device). */
int tlr_ctx_create(int device, tlr_ctx **out);

/* Destroy a context; frees its workspace.  NULL is ignored. */
void tlr_ctx_destroy(tlr_ctx *ctx);

/* Rank buckets of the compression (Sec. 2: the tiles of a column have uneven
 * ranks).  Every tile is compressed from a random sample of s columns, s the
 * tile's rank at the previous evaluation plus an oversampling margin; the
 * QR and SVD stages of a tile run on a thread-block cluster whose size comes
 * from the bucket s falls in: the first b with s <= qr_edge[b] (svd_edge[b]),
 * entry 3 catching all larger s (its edge is ignored).  Tiles of one bucket
 * share one launch.  Sizes are CTAs per cluster: 1, 2, 4, 8 or 16 (16 where
 * the device runs clusters of 16, else 8; a size whose panel does not fit in
 * shared memory grows to the next).  Larger clusters shorten one tile's
 * compression (fewer rows per CTA), smaller ones need fewer SMs per tile and
 * fewer barriers per flop: a single factorisation wants the first, many
 * concurrent ones may want the second (tlr_pool_autotune).  The buckets
 * change how the tile's QR and SVD are reduced, not what they compute: the
 * results agree to rounding.  Default: QR s <= 64 -> 4, <= 128 -> 8, else
 * 16; SVD s <= 48 -> 1, <= 96 -> 4, <= 160 -> 8, else 16. */
typedef struct {
    int32_t qr_edge[4];
    int32_t qr_size[4];
    int32_t svd_edge[4];
    int32_t svd_size[4];
} tlr_buckets;

/* Set the context's rank buckets (NULL restores the default); applies to the
 * calls that start after it.  Errors: TLR_ERR_ARG (a size not in {1, 2, 4, 8,
 * 16}, or edges 0..2 not positive and nondecreasing). */
int tlr_ctx_set_buckets(tlr_ctx *ctx, const tlr_buckets *b);

/* The context's rank buckets.  Errors: TLR_ERR_ARG (NULL). */
int tlr_ctx_get_buckets(const tlr_ctx *ctx, tlr_buckets *out);

/* Message of the last failing call on `ctx` ("" if none).  Owned by ctx. */
const char *tlr_last_error(const tlr_ctx *ctx);

/* Library version string, e.g. "tlr-gb300 0.1 sm_103a". */
const char *tlr_version(void);

/* Number of CUDA kernels the library has launched since it was loaded (all
 * contexts); the difference across a region counts its launches. */
int64_t tlr_launch_count(void);

/* ---- a1: spatial ordering (Sec. 3) -------------------------------------- */

/* Order n locations.  Sec. 3.1 (encode, sort, decode), Sec. 3.2 (KD-tree),
 * Sec. 3.3.1 (max-min), Sec. 5.1 (no order).
 *   xy      device, 2n doubles, SoA; for MORTON/HILBERT each coordinate is
 *           clamped to [0, 1] and quantised as round(v * 65535), ties to even
 *   method  TLR_ORDER_*; seed is used by RANDOM only
 *   perm    device, n int64 (output): position k holds original point perm[k]
 *   codes   device, n uint32 (output, may be NULL): the sort keys of RANDOM,
 *           MORTON and HILBERT in original order; left untouched otherwise
 *   xy_out  device, 2n doubles (output, may be NULL): the permuted locations;
 *           with flags & TLR_ORDER_QUANTIZE the decoded values q / 65535
 * Ties are broken by original index; the result is bit-identical across runs.
 * Errors: TLR_ERR_ARG (n < 0, bad method/flags, NULL perm with n > 0). */
int tlr_order(tlr_ctx *ctx, const double *xy, int64_t n, int method, uint64_t seed,
              uint32_t flags, int64_t *perm, uint32_t *codes, double *xy_out, void *stream);

/* The same ordering as tlr_order for RANDOM, MORTON and HILBERT, for callers
 * that cannot allocate device memory while they run (for instance a serving
 * loop that cannot afford cudaMalloc's implicit device synchronisation, or a
 * process whose device memory is fixed at start-up).  The paper has no
 * counterpart; this is an engineering variant of the Sec. 3.1 pipeline.
 *   xy, n, method, seed, perm, codes: as for tlr_order (device pointers;
 *   codes may be NULL).  No context: the current CUDA device is used.
 * It calls no cudaMalloc / cudaFree: its sort buffers live in one file-scope
 * __device__ array of 4.26 MB that every device loading the library holds
 * until the process exits, so n is limited to 262,144 (2^18) locations.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * previous call's contents (every value a call reads it writes first):
 * calls whose kernels overlap on the GPU race, so issue them on one stream
 * or order them.
 * Errors: TLR_ERR_ARG (n < 0, n > 262144, another method, NULL pointers),
 * TLR_ERR_CUDA (symbol lookup or launch failure). */
int tlr_order_noalloc(const double *xy, int64_t n, int method, uint64_t seed, int64_t *perm,
                      uint32_t *codes, void *stream);

/* dst[k] = src[perm[k]] for k < n (device pointers; permutes Z like the
 * locations).  Errors: TLR_ERR_ARG. */
int tlr_gather(tlr_ctx *ctx, const int64_t *perm, const double *src, int64_t n, double *dst,
               void *stream);

/* ---- a2: covariance tiles (Eq. 1.1, Eq. 4.2) ---------------------------- */

/* Number of doubles of the packed lower-triangular tile array of tlr_generate:
 * NT (NT + 1) / 2 * nb * nb. */
int64_t tlr_tiles_size(int64_t n, int nb);

/* Dense lower-triangular covariance tiles Sigma_ij = C(|s_i - s_j|; theta),
 * i >= j, of the (already ordered) locations xy (device, SoA).  Tile (i, j)
 * starts at tiles + (i (i + 1) / 2 + j) nb^2, column major with leading
 * dimension nb; rows/columns past m_i/m_j are set to 0.  K_nu is evaluated on
 * the device (Temme's series for x <= 2, a continued fraction with the
 * Wronskian for 2 < x <= 25, the asymptotic expansion beyond).
 * Errors: TLR_ERR_ARG (n <= 0, nb out of range, theta not positive). */
int tlr_generate(tlr_ctx *ctx, const double *xy, int64_t n, int nb, tlr_theta theta,
                 double *tiles, void *stream);

/* Product of the mixed-precision path on the tensor cores (tcgen05):
 * C = alpha op(A) op(B) + beta C, op(X) = X or X' (trans_* != 0; not both),
 * all matrices FP64 column major on the device, op(A) m x k, op(B) k x n.
 * Every operand is split into `slices` BF16 slices with a power-of-two scale
 * per row and 64-wide chunk of the inner dimension (error-free splitting of
 * Ozaki, Ogita and Oishi 2012); slice products accumulate in FP32 in tensor
 * memory, and are summed in float-float registers.  slices = 5: about 40
 * significant bits relative to max |a| max |b| of each chunk (the product of
 * the mixed path, TLR_PREC_TENSOR); slices = 1: the plain BF16 product with
 * FP32 accumulation (8 bits).  A test and measurement hook of the kernel the
 * likelihood uses; it allocates split copies of A and B (stream ordered) and
 * returns after the product has finished (it syncs `stream`).
 * Errors: TLR_ERR_ARG (sizes, leading dimensions, slices), TLR_ERR_CUDA (no
 * sm_103a device), TLR_ERR_TIMEOUT (a pipeline wait gave up after 4 s). */
int tlr_gemm_tc(tlr_ctx *ctx, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                int64_t ldc, int slices, void *stream);

/* Matern covariance for m distances (device in, device out); a probe of the
 * device K_nu used by tlr_generate.  Errors: TLR_ERR_ARG. */
int tlr_matern(tlr_ctx *ctx, const double *d, int64_t m, tlr_theta theta, double *out,
               void *stream);

/* ---- TLR matrices ---------------------------------------------------------- */

/* Allocate a TLR matrix for n points, tile nb, off-diagonal capacity maxrank
 * (<= 0: nb / 2).  Device storage: diagonal tiles NT nb^2 doubles; U and V
 * each NT (NT - 1) / 2 * nb * maxrank doubles; ranks NT^2 int32.
 * Errors: TLR_ERR_ARG, TLR_ERR_OOM. */
int tlr_mat_create(tlr_ctx *ctx, int64_t n, int nb, int maxrank, tlr_mat **out);

/* The same matrix with storage sized by a rank map (the TLR memory saving of
 * Sec. 2 and Table 1 made real on the device): rank_map (host, NT x NT row
 * major, r_ij at i NT + j for i > j; e.g. from tlr_mat_ranks of an earlier
 * factor of the same locations) gives each off-diagonal tile
 * min(maxrank, r + max(8, r / 4) rounded up to 8) columns of U and V, plus a
 * shared overflow area of max(sum / 8, 4 maxrank) columns.  A later
 * compression or factorisation whose rank for a tile exceeds its slot moves
 * the tile into the overflow area; if that is full it fails with
 * TLR_ERR_RANK (message: "its slot").  The map also seeds the compression's
 * sample sizes, as the previous factor does for tlr_loglik.
 * Errors: TLR_ERR_ARG, TLR_ERR_OOM. */
int tlr_mat_create_compact(tlr_ctx *ctx, int64_t n, int nb, int maxrank, const int32_t *rank_map,
                           tlr_mat **out);

/* Device bytes held by a TLR matrix (D, U, V, rank map); 0 for NULL. */
int64_t tlr_mat_bytes(const tlr_mat *mat);

/* Host only: the bytes tlr_mat_create (rank_map NULL) or
 * tlr_mat_create_compact would allocate; -1 for invalid sizes. */
int64_t tlr_mat_plan_bytes(int64_t n, int nb, int maxrank, const int32_t *rank_map);

void tlr_mat_destroy(tlr_mat *mat);

/* Device pointers and layout of a TLR matrix (any output may be NULL).
 *   D      diagonal tile t at D + t nb^2 (column major, ld nb; lower triangle
 *          holds L_tt after a factorisation)
 *   U, V   off-diagonal tile (i, j), i > j, index k = i (i - 1) / 2 + j:
 *          for tlr_mat_create, U_k at U + k nb maxrank, V_k at V + k nb maxrank,
 *          column major with ld nb, r_ij valid columns; A_ij ~ U_k V_k'
 *          (a compact matrix places tiles by its own map: use tlr_mat_tile)
 *   ranks  device int32 NT x NT row major; ranks[i NT + j] = r_ij (symmetric),
 *          the diagonal holds m_t */
int tlr_mat_layout(const tlr_mat *mat, int64_t *n, int *nb, int *nt, int *maxrank,
                   double **D, double **U, double **V, int32_t **ranks);

/* Copy one tile to caller buffers (device, column major, ld nb): for i == j
 * the diagonal tile into `a` (nb x nb); for i > j the factors U_ij into `a`
 * and V_ij into `b` (nb x r each; the buffers hold nb x maxrank).  *rank (host)
 * receives r_ij (m_i for i == j).  Stream ordered on `stream`.
 * Errors: TLR_ERR_ARG (i < j, out of range, NULL buffers). */
int tlr_mat_tile(tlr_ctx *ctx, const tlr_mat *mat, int i, int j, double *a, double *b,
                 int32_t *rank, void *stream);

/* Copy the NT x NT rank map to host memory (row major).  Syncs the context's
 * internal copy stream.  Errors: TLR_ERR_ARG, TLR_ERR_CUDA. */
int tlr_mat_ranks(tlr_ctx *ctx, const tlr_mat *mat, int32_t *host_ranks);

/* ---- a3: per-tile compression (Sec. 2, Sec. 3) -------------------------- */

/* Compress the packed dense tiles of tlr_generate into `A`: diagonal tiles are
 * copied, each off-diagonal tile is replaced by U V' with
 * r = #{ singular values > eps_abs } (absolute threshold, normally
 * eps * sigma2).  Randomised range finder with adaptive sample size, then an
 * exact SVD of the projected tile.
 * Errors: TLR_ERR_ARG; TLR_ERR_RANK if some r > maxrank (info = i NT + j). */
int tlr_compress(tlr_ctx *ctx, const double *tiles, int64_t n, int nb, double eps_abs,
                 tlr_mat *A, int64_t *info, void *stream);

/* ---- a4: TLR Cholesky (Sec. 2, Sec. 5.3) -------------------------------- */

/* Factor the TLR matrix A = L L' in place (tile algorithm of akbudak2017tile,
 * left-looking): for each column j, every tile (i, j), i >= j, is updated
 * with the low-rank products of the tiles already factored, the diagonal
 * tile gets a dense Cholesky, each off-diagonal tile is recompressed at
 * eps_abs and its V factor solved with L_jj.  On return D holds L_tt and
 * U V' holds L_ij.
 * Errors: TLR_ERR_NOT_SPD (info = global row), TLR_ERR_RANK (info = i NT + j). */
int tlr_potrf(tlr_ctx *ctx, tlr_mat *A, double eps_abs, int64_t *info, void *stream);

/* ---- a5: triangular solve and log-determinant (Eq. 1.2) ------------------ */

/* With L from tlr_potrf: y = L^-1 z (device, n doubles each; y may alias z),
 * *logdet = 2 sum log L_ii, *quad = y'y (host doubles).  Syncs `stream`.
 * Errors: TLR_ERR_ARG. */
int tlr_solve(tlr_ctx *ctx, const tlr_mat *L, const double *z, double *y, double *logdet,
              double *quad, void *stream);

/* z = L w for a factor L (device vectors): draws Z ~ N(0, L L') from white
 * noise w.  Errors: TLR_ERR_ARG. */
int tlr_lmul(tlr_ctx *ctx, const tlr_mat *L, const double *w, double *z, void *stream);

/* ---- the hot path: one likelihood evaluation ------------------------------ */

/* l(theta) of Eq. 1.2 for ordered locations xy and observations z (device,
 * both already permuted by tlr_order / tlr_gather).  Runs a2-a5 fused: each
 * tile is generated from the Matern kernel directly inside its update, so the
 * dense covariance never exists as a whole.  `L` (created for n, opts->nb,
 * opts->maxrank) receives the factor and its rank map.  *out is filled on the
 * host; the call syncs `stream`.
 * Errors: TLR_ERR_ARG, TLR_ERR_NOT_SPD, TLR_ERR_RANK, TLR_ERR_OOM, TLR_ERR_CUDA. */
int tlr_loglik(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, tlr_theta theta,
               const tlr_opts *opts, tlr_mat *L, tlr_result *out, void *stream);

/* Several evaluations of Eq. 1.2 advanced together on one context (the
 * batched workload: many datasets whose tiles have uneven ranks, Sec. 2).
 * Entry g evaluates l(theta[g]) for the ordered locations xy[g] and
 * observations z[g] (device, n[g] each, as for tlr_loglik) with options
 * opts[g] into L[g] and out[g].  The factorisations run column by column in
 * lockstep, and each step of a column is one launch for all entries: the
 * panel products with the Matern generation, the diagonal POTRF (one
 * cluster per entry), every compression launch class (tiles of all entries
 * bucketed by sample size), V <- L^-1 V, the Gram matrices and the solve.
 * An entry whose factorisation finishes or fails drops out; the others go
 * on.  Every entry's result is bit for bit what tlr_loglik returns for it
 * alone (same L[g] rank map), including the TLR_PREC_AUTO choices.
 *   count   1..32 entries; every entry has its own L[g]
 *   opts    count options; all with the same precision (eps, nb, maxrank
 *           per entry; opts[g].nb == L[g]'s tile size)
 *   out     count results (host); ms_total is the device time of the whole
 *           call (plus, under AUTO, of the call's mixed attempt)
 *   status  count codes (host, may be NULL): TLR_OK, TLR_ERR_NOT_SPD,
 *           TLR_ERR_RANK or TLR_ERR_NAN per entry (out[g].info as for
 *           tlr_loglik); another error stops the call and is written to
 *           every entry
 * Returns TLR_OK, else the first failing entry's status (its message in
 * tlr_last_error).  Syncs `stream`.  Errors: TLR_ERR_ARG, TLR_ERR_NOT_SPD,
 * TLR_ERR_RANK, TLR_ERR_NAN, TLR_ERR_OOM, TLR_ERR_CUDA. */
int tlr_loglik_batch(tlr_ctx *ctx, int count, const double *const *xy, const double *const *z, const int64_t *n,
                     const tlr_theta *theta, const tlr_opts *opts, tlr_mat *const *L, tlr_result *out,
                     int *status, void *stream);

/* The same evaluation from HOST buffers (Sec. 3 + Eq. 1.2 in one call): xy_host
 * (2n doubles, SoA, generation order, in [0,1]^2) and z_host (n doubles, the
 * same order) are copied to the device on `stream` (pinned memory makes the
 * copies asynchronous; pageable memory works too), the locations are ordered
 * by `order` (TLR_ORDER_*; seed for TLR_ORDER_RANDOM), locations and
 * observations permuted, and l(theta) evaluated as tlr_loglik does.  The
 * device copies are workspaces of the call.  *out is filled on the host; the
 * call syncs `stream`.  Errors: those of tlr_order and tlr_loglik. */
int tlr_loglik_host(tlr_ctx *ctx, const double *xy_host, const double *z_host, int64_t n, int order,
                    uint64_t seed, tlr_theta theta, const tlr_opts *opts, tlr_mat *L, tlr_result *out,
                    void *stream);

/* ---- measurement ------------------------------------------------------------ */

/* Enable (enable != 0) or disable CUDA-event timing of the panel update GEMMs
 * (the dominant kernel of tlr_loglik), and read the figures of the last
 * tlr_loglik call: their summed device time (ms), their FP64 flop count, the
 * number of covariance entries their epilogues evaluated and the number of
 * launches.  Any output may be NULL.  Errors: TLR_ERR_ARG (ctx NULL). */
int tlr_profile(tlr_ctx *ctx, int enable, double *gemm_ms, double *gemm_flops,
                double *matern_entries, int *panel_launches);

/* Per-stage device time (ms) of the last profiled tlr_loglik factorisation,
 * summed over all columns, written to ms[0..4]: building the low-rank update
 * operands, the panel update GEMM (with Matern generation), the dense POTRF of
 * the diagonal tile, the compression of the off-diagonal tiles, and the TRSM
 * of their V factors.  Errors: TLR_ERR_ARG. */
int tlr_stage_times(tlr_ctx *ctx, double *ms);

/* Finer device times (ms) of the last profiled tlr_loglik factorisation,
 * summed over columns, written to ms[0..count-1].  Main stream: operands of a
 * main-stream panel update, look-ahead correction by the previous column,
 * wait for the look-ahead stream, forward-solve update, paired-FP32 copy of
 * the panel, main-stream panel GEMM, diagonal copy, compression, wait for the
 * side stream, V <- L^-1 V, solve and log-determinant terms, Gram matrix V'V
 * of the finished column.  Side stream: POTRF, L^-1.  Look-ahead stream:
 * operands and panel GEMM of the next column's update.
 * Returns the number of values written (at most 16), or TLR_ERR_ARG (< 0). */
int tlr_detail_times(tlr_ctx *ctx, double *ms, int count);

/* Device time (ms) of the compression sub-steps of the last profiled
 * factorisation, written to ms[0..6]: sampling GEMM (T Omega), QR of the
 * sample, projection GEMM (T' Q), QR of the projection, SVD of the small
 * factor, host decision (including the stream sync), U/V GEMMs.
 * Errors: TLR_ERR_ARG. */
int tlr_compress_times(tlr_ctx *ctx, double *ms);

/* Counters of the compressions of the last tlr_compress, tlr_loglik or
 * tlr_potrf call, written to out[0..6]: tile compressions run (a tile redone
 * with a larger sample counts again), adaptive rounds, FP64 Jacobi sweeps
 * summed over the compressions, the largest FP64 sweep count of one
 * compression, FP32 (preconditioning) Jacobi sweeps summed, and the QR and
 * SVD jobs that ran on the global-memory kernels (samples too large for a
 * cluster's shared memory).
 * Collected whether or not profiling is on.  Errors: TLR_ERR_ARG. */
int tlr_compress_stats(tlr_ctx *ctx, int64_t *out);

/* The cluster Jacobi SVD on 16-CTA clusters (the high-rank tiles next to the
 * diagonal) during the last profiled factorisation, written to out[0..3]:
 * device time (ms, CUDA events on its stream, summed over launches), FP64
 * floating-point operations as executed (one FP64 product M J of 2 s^3, the
 * column norms at every FP64 sweep, one dot product per pair checked, one
 * two-column rotation per pair rotated), number of launches, and number of
 * clusters (tiles) over those launches.  Errors: TLR_ERR_ARG. */
int tlr_kernel_stats(tlr_ctx *ctx, double *out);

/* ---- MLE (Sec. 5.1: derivative-free, bound-constrained) ------------------ */

/* Maximise l(theta) over lo <= theta <= hi from theta0 with the Nelder-Mead
 * simplex method in log(theta) (bounds by clamping), stopping when the
 * simplex's spread in l falls below tol * (1 + |l|), when its size in
 * log(theta) falls below 1e-8, or after max_iter evaluations.  L holds the
 * factor of the last evaluated theta on return.
 * Failed evaluations (NOT_SPD, RANK) count as l = -inf.  Outputs on host.
 * Errors: TLR_ERR_ARG, or the first hard error of an evaluation. */
int tlr_mle(tlr_ctx *ctx, const double *xy, const double *z, int64_t n, const tlr_opts *opts,
            tlr_theta theta0, tlr_theta lo, tlr_theta hi, double tol, int max_iter,
            tlr_mat *L, tlr_theta *theta_hat, double *ll_hat, int *iters, void *stream);

/* ---- many datasets: batched evaluation and serving -------------------------
 *
 * The paper evaluates each replicate separately (Sec. 5.1); a pool evaluates
 * many independent likelihoods at once.  It keeps datasets resident on one
 * device -- ordered locations, ordered observations, the permutation, and the
 * rank map of each dataset's last factor -- and runs l(theta) requests on
 * `workers` concurrent workers, each a host thread with its own context and
 * streams, so that the kernels of different requests overlap on the device.
 *
 * Admission (continuous batching).  Requests queue in arrival order.  A
 * request starts as soon as a worker is free, no earlier request of its
 * dataset is running, and the device memory it needs fits the pool's HBM
 * budget: its dataset's TLR factor storage (kept resident between requests;
 * idle factors of other datasets are evicted least recently used first when
 * room is needed) plus the evaluation's workspace.  A request waiting for
 * memory to allocate a factor is not overtaken by later requests that would
 * allocate one too.
 *
 * Determinism.  The requests of one dataset run one at a time in submission
 * order, and each starts from the rank map its dataset's previous request
 * left (the sample sizes of the compression, Sec. 2).  The k-th result of a
 * dataset is therefore bit-for-bit the one a single context gets from k
 * tlr_loglik calls on one tlr_mat in that order, whatever else runs beside it.
 *
 * Thread safety: every tlr_pool_* call may be made from any host thread.
 * Errors of a pool call leave a message in tlr_pool_last_error(), kept per
 * calling thread. */
typedef struct tlr_pool tlr_pool;

typedef struct {
    int32_t workers;    /* concurrent evaluations, 1..64 */
    int32_t nb;         /* tile size of datasets added with nb <= 0 (16..1024) */
    int32_t maxrank;    /* off-diagonal rank slots per tile, capped at each dataset's
                           tile size; <= 0 selects half the tile size */
    uint32_t flags;     /* reserved, 0 */
    int64_t hbm_budget; /* device bytes the pool may hold (resident data, factors,
                           workspace); <= 0 selects 90% of the free memory */
} tlr_pool_opts;

/* Create a pool on CUDA device `device`.
 * Errors: TLR_ERR_ARG, TLR_ERR_CUDA, TLR_ERR_OOM. */
int tlr_pool_create(int device, const tlr_pool_opts *opts, tlr_pool **out);

/* Finish every queued request, stop the workers and free the pool's memory.
 * Results not yet collected by tlr_pool_wait are discarded.  No other call
 * on the pool may run concurrently with it or follow it.  NULL is ignored. */
void tlr_pool_destroy(tlr_pool *p);

/* Message of the last failing tlr_pool_* call of the calling thread. */
const char *tlr_pool_last_error(void);

/* Register a dataset of n locations xy (SoA, 2n values) and observations z
 * (n values); both host or device pointers, copied.  The locations are
 * ordered on the device with `order` (TLR_ORDER_*, `seed` for RANDOM) and
 * the observations permuted alike; the dataset's tile size is nb (<= 0: the
 * pool's).  *id receives its handle.
 * Errors: TLR_ERR_ARG; TLR_ERR_OOM if its resident bytes, plus the factor and
 * workspace of the largest registered dataset, would exceed the budget. */
int tlr_pool_add(tlr_pool *p, const double *xy, const double *z, int64_t n, int order, uint64_t seed,
                 int nb, int *id);

/* Wait for the dataset's queued requests, then unregister it and free its
 * memory.  Errors: TLR_ERR_ARG (unknown id). */
int tlr_pool_remove(tlr_pool *p, int id);

/* Device pointers of a dataset's resident data (any output may be NULL): n,
 * tile size, ordered locations (2n), ordered observations (n), permutation
 * (n, position -> input index), and the largest rank of its last factor (0
 * before the first evaluation).  Pointers stay valid until the dataset is
 * removed; read them only while no request of the dataset runs.
 * Errors: TLR_ERR_ARG. */
int tlr_pool_dataset(tlr_pool *p, int id, int64_t *n, int *nb, const double **xy, const double **z,
                     const int64_t **perm, int32_t *last_max_rank);

/* Queue one l(theta) evaluation (Eq. 1.2) of dataset `id` at accuracy eps
 * (tlr_opts.eps) and precision TLR_PREC_*; returns at once with *ticket.
 * Errors: TLR_ERR_ARG (unknown id, bad eps/precision). */
int tlr_pool_submit(tlr_pool *p, int id, tlr_theta theta, double eps, int precision, int64_t *ticket);

/* Block until request `ticket` has finished; its result goes to *out (may be
 * NULL) and, if times_ms is not NULL, times_ms[0..2] = time queued, time
 * running, and latency from submission to completion (host clock, ms).  The
 * ticket is consumed.  Returns the request's own status (a failed
 * evaluation's message is then in tlr_pool_last_error()), or TLR_ERR_ARG for
 * an unknown ticket. */
int tlr_pool_wait(tlr_pool *p, int64_t ticket, tlr_result *out, double *times_ms);

/* Batched evaluation: submit count requests (ids[i], theta[i]) and wait for
 * all of them.  out[i] and status[i] (either may be NULL) receive each
 * result; returns TLR_OK if all succeeded, else the first failing status in
 * index order. */
int tlr_pool_loglik(tlr_pool *p, int count, const int *ids, const tlr_theta *theta, double eps,
                    int precision, tlr_result *out, int *status);

/* tlr_mle (the same search and stopping rules) for a resident dataset, run
 * on the calling thread with every evaluation submitted to the pool, where it
 * mixes with the other requests.  Outputs on host. */
int tlr_pool_mle(tlr_pool *p, int id, double eps, int precision, tlr_theta theta0, tlr_theta lo,
                 tlr_theta hi, double tol, int max_iter, tlr_theta *theta_hat, double *ll_hat, int *iters);

/* Tile-size autotuning for one dataset: for each candidate tile size
 * cands[0..ncand) that fits the budget, two evaluations at theta (the first
 * sets the rank map, the second is timed on the device); the dataset keeps
 * the fastest tile size, written to *best, with ms[i] the timed evaluation
 * (-1 if skipped).  The dataset's rank map restarts empty.  Waits for the
 * dataset's queued requests first.  Errors: TLR_ERR_ARG, or the first error
 * of an evaluation. */
int tlr_pool_tune(tlr_pool *p, int id, tlr_theta theta, double eps, int precision, const int32_t *cands,
                  int ncand, int32_t *best, double *ms);

/* Batched launches and rank buckets of the pool's workers.  group (1..32):
 * a worker that admits a request also admits, up to `group` in all, the
 * queued requests of the same precision that can start now (each under the
 * admission rules above, in queue order), and evaluates them together with
 * tlr_loglik_batch: each step of their factorisations' tile columns is one
 * launch for all of them.  buckets (NULL: the default) become the rank
 * buckets (tlr_ctx_set_buckets) of every worker's context.  Applies to
 * requests admitted after the call; results do not depend on group (every
 * result is the one tlr_loglik gives), and the buckets change them only by
 * rounding.  Default: group 1, default buckets.  Errors: TLR_ERR_ARG. */
int tlr_pool_configure(tlr_pool *p, int group, const tlr_buckets *buckets);

/* The pool's current group size and buckets (either output may be NULL). */
int tlr_pool_get_config(tlr_pool *p, int *group, tlr_buckets *buckets);

/* Throughput autotuner of the batched workload (rank-bucket and group-size
 * tuning): the `count` requests (ids[i], theta[i]) at eps / precision are
 * evaluated once at the current configuration (which also sets the rank
 * maps every candidate then starts from), then `rounds` times under each
 * candidate c (group size groups[c], buckets[c]; buckets NULL keeps the
 * current buckets), timed on the host clock from the first submission to
 * the last result.  evals_per_s[c] (may be NULL) receives each candidate's
 * successful evaluations per second; the pool keeps the fastest candidate,
 * whose index goes to *best.  The datasets keep the rank maps of their last
 * evaluation.  Errors: TLR_ERR_ARG (bad candidates or unknown datasets). */
int tlr_pool_autotune(tlr_pool *p, int count, const int *ids, const tlr_theta *theta, double eps, int precision,
                      int ncand, const int32_t *groups, const tlr_buckets *buckets, int rounds,
                      double *evals_per_s, int *best);

/* Device bytes the admission model charges for a dataset of n locations at
 * tile size nb and rank slots maxrank (<= 0: nb / 2), written to out[0..2]:
 * resident data (32 n: locations, observations, permutation), TLR factor
 * storage (NT nb^2 diagonal + 2 nb maxrank per off-diagonal tile, doubles,
 * plus the NT^2 int32 rank map), and the estimated workspace of one
 * evaluation before the dataset's first rank map is known.  Host only.
 * Errors: TLR_ERR_ARG. */
int tlr_pool_footprint(int64_t n, int nb, int maxrank, int64_t *out);

/* Counters, written to out[0..count) (returns the number written, at most
 * 14): budget, bytes in use, peak bytes in use, resident dataset bytes,
 * resident factor bytes, resident factors, evictions, requests completed,
 * requests queued, requests running, most requests running at once, factor
 * allocations, group evaluations run (more than one request), requests
 * those held.  Byte figures follow the admission model (factor storage
 * exact, workspace estimated). */
int tlr_pool_stats(tlr_pool *p, int64_t *out, int count);

/* Placement of datasets on the GPUs of a job (the batched and served
 * workloads shard by dataset; no collective on the data path): dataset i,
 * of HBM footprint bytes[i] (tlr_pool_footprint: resident data + factor +
 * workspace), goes to rank_of[i] in 0..nranks-1.  Largest footprint first
 * (ties: lower index), each onto the rank with the least bytes placed so far
 * (ties: lower rank) among those whose budget[r] (NULL: unlimited) still has
 * room: the longest-processing-time rule, whose heaviest rank carries at most
 * 4/3 of the optimum when cost follows bytes (Graham 1969).  Deterministic:
 * every rank computes the same placement without communicating.  Host only.
 * Errors: TLR_ERR_ARG; TLR_ERR_OOM if some dataset fits no rank. */
int tlr_shard_place(int count, const int64_t *bytes, int nranks, const int64_t *budget, int32_t *rank_of);

/* The admission policy of the pool run as a discrete-event simulation on the
 * host (no device used): `workers` slots, `ndata` datasets with base, factor
 * and workspace bytes, and nreq requests (dataset req_data[i], arriving at
 * req_arrival[i], nondecreasing, and running for req_cost[i] once started).
 * Writes each request's start and finish time, the peak bytes in use and the
 * number of evictions.  Errors: TLR_ERR_ARG; TLR_ERR_OOM if some dataset
 * could not be registered under the budget. */
int tlr_sched_simulate(int64_t budget, int workers, int ndata, const int64_t *base_bytes,
                       const int64_t *factor_bytes, const int64_t *work_bytes, int nreq,
                       const int32_t *req_data, const double *req_arrival, const double *req_cost,
                       double *start, double *finish, int64_t *peak_bytes, int64_t *evictions);

#ifdef __cplusplus
}
#endif

#endif /* TLR_H */

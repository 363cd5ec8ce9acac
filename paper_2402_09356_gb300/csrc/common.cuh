// Internal definitions shared by the CUDA translation units of the TLR library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <utility>
#include <string>
#include <vector>

#include "../../include/tlr.h"

namespace tlr {

// Device-side status word: the first failing kernel wins the atomicCAS on
// `code`; `info` carries the failing row / tile.
struct DevStatus {
    int code;
    int pad;
    long long info;
};

__device__ inline void set_status(DevStatus *st, int code, long long info) {
    if (atomicCAS(&st->code, 0, code) == 0) st->info = info;
}

// Error carried back to the C ABI.
struct Error {
    int code;
    std::string msg;
};

#define TLR_CUDA_TRY(expr)                                                               \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            throw ::tlr::Error{e_ == cudaErrorMemoryAllocation ? TLR_ERR_OOM : TLR_ERR_CUDA, \
                               std::string(#expr) + ": " + cudaGetErrorString(e_)};     \
    } while (0)

#define TLR_CHECK_LAUNCH() TLR_CUDA_TRY(cudaGetLastError())

inline Error make_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return Error{code, buf};
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Most factorisations advanced together in one call (tlr_loglik_batch).
constexpr int kMaxGroup = 32;

// Rank buckets of the compression (tlr_buckets): entries per table, default.
constexpr int kBuckets = 4;
inline tlr_buckets default_buckets() {
    return tlr_buckets{{64, 128, INT32_MAX, INT32_MAX}, {4, 8, 16, 16}, {48, 96, 160, INT32_MAX}, {1, 4, 8, 16}};
}
inline bool buckets_ok(const tlr_buckets &b) {
    auto size_ok = [](int32_t c) { return c == 1 || c == 2 || c == 4 || c == 8 || c == 16; };
    for (int k = 0; k < kBuckets; ++k)
        if (!size_ok(b.qr_size[k]) || !size_ok(b.svd_size[k])) return false;
    for (int k = 0; k + 1 < kBuckets - 1; ++k)
        if (b.qr_edge[k] > b.qr_edge[k + 1] || b.svd_edge[k] > b.svd_edge[k + 1]) return false;
    return b.qr_edge[0] > 0 && b.svd_edge[0] > 0;
}

// Number of kernels this library has launched (all contexts, all devices).
extern std::atomic<long long> g_launch_count;

// Every kernel of the library is launched through here so that launches can
// be counted.
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args &&...args) {
    kernel<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
}

// Launch on thread-block clusters of `csize` CTAs (counted like launch()).
template <typename... KArgs, typename... Args>
inline void launch_clustered(void (*kernel)(KArgs...), int csize, int nclusters, int threads, size_t smem,
                             cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * csize));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TLR_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, args...));
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
}

// Stream-ordered device buffer from the CUDA memory pool.
class DevBuf {
public:
    DevBuf() = default;
    DevBuf(size_t bytes, cudaStream_t s) { alloc(bytes, s); }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    void alloc(size_t bytes, cudaStream_t s) {
        release();
        stream_ = s;
        bytes_ = bytes;
        if (bytes) TLR_CUDA_TRY(cudaMallocAsync(&ptr_, bytes, s));
    }
    void release() {
        if (ptr_) cudaFreeAsync(ptr_, stream_);
        ptr_ = nullptr;
        bytes_ = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(ptr_); }
    size_t bytes() const { return bytes_; }

private:
    void *ptr_ = nullptr;
    size_t bytes_ = 0;
    cudaStream_t stream_ = nullptr;
};

// A pinned host ring mirrored in device memory for kernel descriptors.  One
// ring per stream that launches kernels reading descriptors, so that a ring
// is only reset after a sync of the one stream whose kernels read it.
struct StageRing {
    char *h = nullptr;
    char *d = nullptr;
    size_t cap = 0;
    size_t off = 0;
};

}  // namespace tlr

struct tlr_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    tlr::DevStatus *d_status = nullptr;   // device status words: the context's, then one per grouped factorisation
    tlr::DevStatus *h_status = nullptr;   // pinned host mirror
    cudaStream_t aux = nullptr;           // second stream for concurrent tile work (high priority)
    cudaStream_t la = nullptr;            // look-ahead stream: the next column's panel update
    // CTAs per SM the look-ahead panel GEMM may hold (shared memory reserved so
    // that the critical-path kernels keep room); 0 = no reservation (several
    // factorisations sharing the device)
    int ahead_ctas_per_sm = 1;
    cudaEvent_t ev_la_fork = nullptr, ev_la_join = nullptr;
    cudaStream_t hp = nullptr;            // high-priority stream of the factorisation's compression
    cudaStream_t sv = nullptr;            // the fused forward solve, beside the next column's work
    cudaEvent_t ev_sv_fork = nullptr, ev_sv_done = nullptr;
    cudaEvent_t ev_hp_fork = nullptr, ev_hp_join = nullptr;
    // compression: one stream per launch class (cluster size), forked from and
    // joined to the calling stream
    static constexpr int kClassStreams = 4, kClassEvents = 8;
    cudaStream_t cls_stream[kClassStreams] = {};
    cudaEvent_t cls_fork = nullptr, cls_join[kClassEvents] = {};
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_fork = nullptr, ev_join = nullptr;
    // descriptor staging: ring 0 for the caller's stream, 1 for `aux`, 2 for `la`, 3 for `hp`, 4 for `sv`
    tlr::StageRing stage[5];
    // fixed Gaussian test matrices of the randomised range finder
    double *d_omega = nullptr;
    float2 *d_omega2 = nullptr;  // paired-FP32 copy of d_omega
    int omega_rows = 0, omega_cols = 0;
    // per-theta Matern interpolation table (+ node scratch)
    double *d_mtab = nullptr;
    // timing of the dominant kernel (panel update GEMMs)
    bool profile = false;
    std::vector<cudaEvent_t> prof_events;
    double last_gemm_ms = 0.0, last_gemm_flops = 0.0, last_matern_entries = 0.0;
    int last_panel_launches = 0;
    double last_stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double last_detail_ms[16] = {};
    // compression sub-steps (when profiling): sample GEMM, QR of Y, projection
    // GEMM, QR of B', SVD, host decision (incl. sync), U/V GEMMs
    std::vector<cudaEvent_t> comp_events;
    size_t comp_used = 0;                     // events of comp_events recorded since the last collect
    std::vector<cudaEvent_t> comp_pending;    // complete rounds (8 marks each) not yet read
    double comp_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    long long comp_stats[7] = {};  // tiles, rounds, FP64 Jacobi sweeps (sum, max), FP32 sweeps (sum), QR / SVD jobs on the global-memory kernels
    // the 16-CTA cluster Jacobi (profiling): device ms, FP64 flops, launches, clusters
    std::vector<cudaEvent_t> cls_time_events;
    double *d_potrf_scratch = nullptr;  // diagonal-block inverses of the cluster POTRF (per job)
    int potrf_scratch_jobs = 0;
    double k16_ms = 0.0, k16_flops = 0.0;
    long long k16_launches = 0, k16_clusters = 0;
    tlr_buckets buckets = tlr::default_buckets();  // compression launch classes by sample size
};

struct tlr_mat {
    int device = 0;
    int64_t n = 0;
    int nb = 0;
    int nt = 0;
    int maxrank = 0;
    double *D = nullptr;        // nt * nb * nb
    double *U = nullptr;        // uniform: noff * nb * maxrank; compact: (sum cap + arena) * nb
    double *V = nullptr;        // same layout as U
    int32_t *ranks = nullptr;   // nt * nt
    std::vector<int32_t> h_ranks;  // host mirror, refreshed after compress / factor
    // Compact layout (empty vectors: uniform slots of maxrank columns).  Tile k
    // = off_index(i, j) starts at column base_off[k] of U and V with room for
    // cap[k] columns; a factorisation that finds a larger rank moves the tile
    // into the arena (columns arena_off .. arena_off + arena_cols), and off /
    // cur_cap hold where every tile lives in the current factor.
    std::vector<int64_t> base_off, off;
    std::vector<int32_t> cap, cur_cap;
    int64_t arena_off = 0, arena_cols = 0, arena_next = 0;
    bool cap_overflow = false;  // the last factorisation ran out of room (arena full)
    double last_pivot2 = 0.0;   // min_i L_ii^2 / sigma2 of the last likelihood (0: none yet)
    size_t bytes = 0;           // device bytes of D, U, V and the rank map
};

namespace tlr {

inline int stage_ring(const tlr_ctx *ctx, cudaStream_t s) {
    return s == ctx->aux ? 1 : (s == ctx->la ? 2 : (s == ctx->hp ? 3 : (s == ctx->sv ? 4 : 0)));
}
// Marks the ring of stream s empty; only valid right after a sync of s.
inline void stage_reset(tlr_ctx *ctx, cudaStream_t s) { ctx->stage[stage_ring(ctx, s)].off = 0; }

inline int64_t off_index(int i, int j) { return (int64_t)i * (i - 1) / 2 + j; }
// First column of off-diagonal tile (i, j) in U and V, and its capacity.
inline int64_t slot_col(const tlr_mat *M, int i, int j) {
    const int64_t k = off_index(i, j);
    return M->off.empty() ? k * M->maxrank : M->off[(size_t)k];
}
inline int slot_cap(const tlr_mat *M, int i, int j) {
    return M->cur_cap.empty() ? M->maxrank : M->cur_cap[(size_t)off_index(i, j)];
}
inline int tile_rows(int64_t n, int nb, int t) {
    int64_t r = n - (int64_t)t * nb;
    return (int)(r < nb ? r : nb);
}

// Copies `bytes` of host data into the staging ring of stream `s` (one ring
// per internal stream, ring 0 for the caller's) and returns the device address
// of the copy (stream ordered on `s`).
void *stage_push(tlr_ctx *ctx, const void *data, size_t bytes, cudaStream_t s);

// Status word helpers (host side).
void status_reset(tlr_ctx *ctx, cudaStream_t s);
// Copies the status word to the host and syncs `s`; returns the device code.
int status_fetch(tlr_ctx *ctx, cudaStream_t s, long long *info);

}  // namespace tlr

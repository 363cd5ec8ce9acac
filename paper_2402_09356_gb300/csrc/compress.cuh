// Per-tile compression (declarations; see compress.cu).
#pragma once

#include <functional>

#include "common.cuh"

namespace tlr {

constexpr int kMaxTile = 1024;    // largest tile size nb
constexpr int kMaxSample = 512;   // largest randomised sample size

// One dense tile to compress: T (m x k, ld ldt) -> U (m x r, ld ldu), V (k x r, ld ldv).
struct CompressJob {
    const double *T;
    int ldt;
    const float2 *T2;  // paired-FP32 copy of T (same ld), for the mixed-precision products; or null
    int m, k;
    double *U;
    int ldu;
    double *V;
    int ldv;
    int s_guess;        // expected rank (previous evaluation), drives the first sample size
    long long tile_id;  // i * NT + j, reported on failure
    int cap;            // columns of U / V available (<= 0: maxrank)
    double tau;         // absolute accuracy (compress_jobs; compress_tiles sets it)
    int maxrank;        // largest admissible rank (likewise)
    int item;           // factorisation the tile belongs to (several in one call)
};

// Job outcomes of compress_jobs other than a rank.
constexpr int kCompNan = -1;  // the tile holds non-finite values
constexpr int kCompBad = -2;  // rank above maxrank, unresolved within the sample cap, or no room

// Called with a job whose rank r exceeds its capacity but not maxrank: gives
// the job new U / V storage for r columns (same leading dimensions), or
// returns false (the tile is then reported in *bad_tile).
using GrowSlot = std::function<bool(const CompressJob &, int r, double **U, double **V)>;

// Allocate and fill the context's Gaussian test matrix and its paired-FP32
// copy (once).
void ensure_omega(tlr_ctx *ctx, cudaStream_t s);

// Compress every job at absolute accuracy tau.  ranks[q] receives r for job q.
// A tile whose rank exceeds maxrank (or cannot be resolved within the sample
// cap, or exceeds its capacity where `grow` finds no room) is reported in
// *bad_tile (its tile_id), a tile holding non-finite values in *nan_tile;
// both are -1 otherwise.
// With df, the sampling and projection products run in paired-FP32
// arithmetic (every job must then carry T2), and the QR in paired FP32; with
// tc as well, the two products run on the tensor cores (BF16 slices, from
// the FP64 tiles; T2 unused).  `overlap`, if set, is called
// once, after the first round's work is enqueued and before the host waits
// for it (the caller enqueues independent work on other streams there).
// Syncs `s` once per adaptive round.
void compress_tiles(tlr_ctx *ctx, cudaStream_t s, std::vector<CompressJob> &jobs, double tau,
                    int maxrank, std::vector<int> &ranks, long long *bad_tile, long long *nan_tile,
                    bool df = false, const std::function<void()> &overlap = nullptr,
                    const GrowSlot &grow = nullptr, bool tc = false);

// The same for jobs that carry their own tau and maxrank (tiles of several
// factorisations in one call: every launch class serves all of them).
// ranks[q] receives r, or kCompNan / kCompBad; fail_order lists the failed
// jobs in the order their failures were found.
void compress_jobs(tlr_ctx *ctx, cudaStream_t s, std::vector<CompressJob> &jobs, std::vector<int> &ranks,
                   std::vector<int> &fail_order, bool df = false, const std::function<void()> &overlap = nullptr,
                   const GrowSlot &grow = nullptr, bool tc = false);

// Profiling (ctx->profile): compress_jobs records its sub-step marks without
// waiting for them; compress_profile_collect waits for the marks recorded
// since the last reset, adds their intervals to ctx->comp_ms and resets.
// compress_tiles collects by itself; a caller of compress_jobs resets before
// its first call and collects after its last.
void compress_profile_reset(tlr_ctx *ctx);
void compress_profile_collect(tlr_ctx *ctx);

}  // namespace tlr

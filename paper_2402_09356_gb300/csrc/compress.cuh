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
};

// Allocate and fill the context's Gaussian test matrix and its paired-FP32
// copy (once).
void ensure_omega(tlr_ctx *ctx, cudaStream_t s);

// Compress every job at absolute accuracy tau.  ranks[q] receives r for job q.
// A tile whose rank exceeds maxrank (or cannot be resolved within the sample
// cap) is reported in *bad_tile (its tile_id), a tile holding non-finite
// values in *nan_tile; both are -1 otherwise.
// With df, the sampling and projection products run in paired-FP32
// arithmetic (every job must then carry T2).  `overlap`, if set, is called
// once, after the first round's work is enqueued and before the host waits
// for it (the caller enqueues independent work on other streams there).
// Syncs `s` once per adaptive round.
void compress_tiles(tlr_ctx *ctx, cudaStream_t s, std::vector<CompressJob> &jobs, double tau,
                    int maxrank, std::vector<int> &ranks, long long *bad_tile, long long *nan_tile,
                    bool df = false, const std::function<void()> &overlap = nullptr);

}  // namespace tlr

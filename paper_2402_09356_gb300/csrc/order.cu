// a1: spatial ordering of the locations (Sec. 3).
//
// Morton / Hilbert / random: one thread per point computes a 32-bit key
// (Sec. 3.1 "Encoding"), then a stable LSD radix sort orders (key, index)
// pairs (Sec. 3.1 "Sorting"; stability breaks ties by original index).
//
// KD-tree (Sec. 3.2): built level by level.  The segment structure of every
// level depends on n only (a node of m points has children of ceil(m/2) and
// floor(m/2) points), so each level is: per-segment coordinate ranges
// (atomics on order-preserving integer images of the doubles), choice of the
// wider dimension, and one stable radix sort of (segment, rank of the point
// along the chosen dimension).  The ranks come from two initial global sorts
// by (x, index) and (y, index), so sorting by rank inside a segment is sorting
// by (coordinate, index).
//
// Max-min (Sec. 3.3.1): one launch per selected point; every block updates
// the minimum squared distances of its points to the newest selection and
// publishes its (max, lowest index) partial; the next launch reduces the
// partials (double-buffered) to find the next point.  All distance arithmetic
// uses explicitly rounded intrinsics so that no multiply-add is contracted.
#include <mutex>

#include "common.cuh"

namespace tlr {

static constexpr int kSortThreads = 256;
static constexpr int kSortItems = 16;  // keys per thread per block
static constexpr int kSortTile = kSortThreads * kSortItems;

// ---------------------------------------------------------------- key helpers
__device__ __forceinline__ uint32_t quantize16(double v) {
    double c = fmin(fmax(v, 0.0), 1.0);
    return (uint32_t)rint(__dmul_rn(c, 65535.0));  // round half to even
}

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Hilbert index of a cell of the 2^16 x 2^16 grid, orientation of Figure 3:
// quadrants visited lower-left, upper-left, upper-right, lower-right.  The
// frame of the current sub-square is tracked as (swap, complement) flags:
// entering the lower-left quadrant transposes the frame, entering the
// lower-right quadrant transposes and complements it.
__device__ __forceinline__ uint32_t hilbert16(uint32_t qx, uint32_t qy) {
    uint32_t d = 0;
    bool sw = false, cp = false;
#pragma unroll
    for (int b = 15; b >= 0; --b) {
        uint32_t bx = (qx >> b) & 1u, by = (qy >> b) & 1u;
        if (cp) { bx ^= 1u; by ^= 1u; }
        if (sw) { uint32_t t = bx; bx = by; by = t; }
        uint32_t q = (bx << 1) | (bx ^ by);
        d = (d << 2) | q;
        if (q == 0u) sw = !sw;
        else if (q == 3u) { sw = !sw; cp = !cp; }
    }
    return d;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t s) {
    uint64_t z = s + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Order-preserving unsigned image of a double (total order of finite values).
__device__ __forceinline__ uint64_t dkey(double v) {
    uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(uint64_t k) {
    uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

__global__ void k_sfc_keys(const double *__restrict__ xy, int64_t n, int method, uint64_t seed,
                           uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k;
    if (method == TLR_ORDER_RANDOM) {
        k = (uint32_t)(splitmix64(seed ^ (uint64_t)i) >> 32);
    } else {
        uint32_t qx = quantize16(xy[i]), qy = quantize16(xy[n + i]);
        k = (method == TLR_ORDER_MORTON) ? (spread_bits(qx) | (spread_bits(qy) << 1))
                                         : hilbert16(qx, qy);
    }
    keys[i] = k;
    vals[i] = (uint32_t)i;
}

// ------------------------------------------------------------- radix sort
template <typename K>
__global__ void k_radix_hist(const K *__restrict__ keys, int64_t n, int shift,
                             uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortItems; ++c) {
        int64_t i = base + (int64_t)c * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&sh[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = sh[threadIdx.x];
}

// Exclusive scan of `len` uint32 in one block of 1024 threads.
__global__ void k_scan_exclusive(uint32_t *__restrict__ a, int64_t len) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int64_t chunk = (len + 1023) / 1024;
    int64_t lo = t * chunk, hi = lo + chunk < len ? lo + chunk : len;
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan
        uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = t ? part[t - 1] : 0u;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

template <typename K>
__global__ void k_radix_scatter(const K *__restrict__ keys, const uint32_t *__restrict__ vals,
                                int64_t n, int shift, const uint32_t *__restrict__ hist, int nblk,
                                K *__restrict__ keys_out, uint32_t *__restrict__ vals_out) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_cnt[kSortThreads / 32][256];
    __shared__ uint32_t s_tot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = hist[(int64_t)tid * nblk + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortItems; ++c) {
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) s_cnt[w][tid] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)c * kSortThreads + tid;
        bool valid = i < n;
        K k = valid ? keys[i] : K(0);
        uint32_t d = valid ? ((uint32_t)(k >> shift) & 0xFFu) : 0xFFFFFFFFu;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t lower = __popc(peers & ((1u << lane) - 1u));
        if (valid && lower == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t t = s_cnt[w][tid];
            s_cnt[w][tid] = run;
            run += t;
        }
        s_tot[tid] = run;
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[d] + s_cnt[warp][d] + lower;
            keys_out[pos] = k;
            vals_out[pos] = vals[i];
        }
        __syncthreads();
        s_base[tid] += s_tot[tid];
    }
}

// Stable sort of (key, val) pairs by the low `bits` bits of the key.  The
// result ends in (*keys, *vals) (the buffers are swapped as passes proceed).
template <typename K>
static void radix_sort(K **keys, uint32_t **vals, K **keys_tmp, uint32_t **vals_tmp, int64_t n,
                       int bits, uint32_t *hist, cudaStream_t s) {
    if (n <= 1) return;
    int nblk = (int)ceil_div(n, kSortTile);
    for (int shift = 0; shift < bits; shift += 8) {
        launch(k_radix_hist<K>, nblk, kSortThreads, 0, s, *keys, n, shift, hist, nblk);
        launch(k_scan_exclusive, 1, 1024, 0, s, hist, (int64_t)256 * nblk);
        launch(k_radix_scatter<K>, nblk, kSortThreads, 0, s, *keys, *vals, n, shift, hist, nblk,
                                                          *keys_tmp, *vals_tmp);
        TLR_CHECK_LAUNCH();
        std::swap(*keys, *keys_tmp);
        std::swap(*vals, *vals_tmp);
    }
}

static size_t hist_words(int64_t n) { return (size_t)256 * (size_t)ceil_div(n > 0 ? n : 1, kSortTile); }

// ------------------------------------------------------------- outputs
__global__ void k_perm_out(const uint32_t *__restrict__ vals, int64_t n, int64_t *__restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int64_t)vals[i];
}

__global__ void k_iota32(int64_t n, uint32_t *__restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_iota(int64_t n, int64_t *__restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = i;
}

__global__ void k_permute_xy(const double *__restrict__ xy, const int64_t *__restrict__ perm,
                             int64_t n, int quantize, double *__restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    double x = xy[p], y = xy[n + p];
    if (quantize) {
        x = __ddiv_rn((double)quantize16(x), 65535.0);
        y = __ddiv_rn((double)quantize16(y), 65535.0);
    }
    out[k] = x;
    out[n + k] = y;
}

__global__ void k_gather(const int64_t *__restrict__ perm, const double *__restrict__ src,
                         int64_t n, double *__restrict__ dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    dst[k] = (p >= 0 && p < n) ? src[p] : __longlong_as_double(0x7FF8000000000000ll);
}

// ------------------------------------------------------------- KD-tree
__global__ void k_coord_keys(const double *__restrict__ c, int64_t n, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = dkey(c[i]);
    vals[i] = (uint32_t)i;
}

// rank[vals[p]] = p: the position of each point in the (coordinate, index) order
__global__ void k_invert(const uint32_t *__restrict__ vals, int64_t n, uint32_t *__restrict__ rank) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) rank[vals[p]] = (uint32_t)p;
}

__device__ __forceinline__ int seg_of(const int64_t *__restrict__ starts, int nseg, int64_t p) {
    int lo = 0, hi = nseg - 1;  // last start <= p
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_kd_init_ranges(int nseg, unsigned long long *__restrict__ rng) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    rng[4 * s + 0] = ~0ull;  // min x
    rng[4 * s + 1] = 0ull;   // max x
    rng[4 * s + 2] = ~0ull;  // min y
    rng[4 * s + 3] = 0ull;   // max y
}

__global__ void k_kd_ranges(const double *__restrict__ xy, int64_t n, const uint32_t *__restrict__ order,
                            const int64_t *__restrict__ starts, int nseg,
                            unsigned long long *__restrict__ rng) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int s = seg_of(starts, nseg, p);
    uint32_t i = order[p];
    unsigned long long kx = dkey(xy[i]), ky = dkey(xy[n + i]);
    atomicMin(&rng[4 * s + 0], kx);
    atomicMax(&rng[4 * s + 1], kx);
    atomicMin(&rng[4 * s + 2], ky);
    atomicMax(&rng[4 * s + 3], ky);
}

__global__ void k_kd_keys(int64_t n, const uint32_t *__restrict__ order, const int64_t *__restrict__ starts,
                          int nseg, const unsigned long long *__restrict__ rng,
                          const uint32_t *__restrict__ rank_x, const uint32_t *__restrict__ rank_y,
                          int rbits, uint64_t *__restrict__ keys) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int s = seg_of(starts, nseg, p);
    double rx = __dsub_rn(dkey_inv(rng[4 * s + 1]), dkey_inv(rng[4 * s + 0]));
    double ry = __dsub_rn(dkey_inv(rng[4 * s + 3]), dkey_inv(rng[4 * s + 2]));
    uint32_t i = order[p];
    uint32_t r = (rx >= ry) ? rank_x[i] : rank_y[i];  // equal ranges: x
    keys[p] = ((uint64_t)s << rbits) | (uint64_t)r;
}

// ------------------------------------------------------------- max-min
__device__ __forceinline__ double sqdist(double ax, double ay, double bx, double by) {
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

struct MaxLoc {
    double v;
    long long i;
};

__device__ __forceinline__ bool better_max(double v, long long i, double bv, long long bi) {
    return v > bv || (v == bv && i < bi);
}
__device__ __forceinline__ bool better_min(double v, long long i, double bv, long long bi) {
    return v < bv || (v == bv && i < bi);
}

// Block reduction of (value, index) pairs; `is_max` picks max (else min),
// ties to the lower index.  Result valid in thread 0.
__device__ MaxLoc block_argext(double v, long long i, bool is_max) {
    __shared__ double sv[32];
    __shared__ long long si[32];
    for (int off = 16; off; off >>= 1) {
        double ov = __shfl_down_sync(0xFFFFFFFFu, v, off);
        long long oi = __shfl_down_sync(0xFFFFFFFFu, i, off);
        if (is_max ? better_max(ov, oi, v, i) : better_min(ov, oi, v, i)) { v = ov; i = oi; }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) { sv[w] = v; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? sv[lane] : (is_max ? -INFINITY : INFINITY);
        i = lane < nw ? si[lane] : 0x7FFFFFFFFFFFFFFFll;
        for (int off = 16; off; off >>= 1) {
            double ov = __shfl_down_sync(0xFFFFFFFFu, v, off);
            long long oi = __shfl_down_sync(0xFFFFFFFFu, i, off);
            if (is_max ? better_max(ov, oi, v, i) : better_min(ov, oi, v, i)) { v = ov; i = oi; }
        }
    }
    return MaxLoc{v, i};
}

// Bounding box of all points (one block; grid-stride).
__global__ void k_bbox(const double *__restrict__ xy, int64_t n, double *__restrict__ bbox) {
    double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double x = xy[i], y = xy[n + i];
        mnx = fmin(mnx, x); mxx = fmax(mxx, x);
        mny = fmin(mny, y); mxy = fmax(mxy, y);
    }
    MaxLoc a = block_argext(-mnx, 0, true);
    double r0 = -a.v;
    __syncthreads();
    MaxLoc b = block_argext(mxx, 0, true);
    __syncthreads();
    MaxLoc c = block_argext(-mny, 0, true);
    __syncthreads();
    MaxLoc d = block_argext(mxy, 0, true);
    if (threadIdx.x == 0) {
        bbox[0] = __dmul_rn(__dadd_rn(r0, b.v), 0.5);
        bbox[1] = __dmul_rn(__dadd_rn(-c.v, d.v), 0.5);
    }
}

// First point: nearest to the bounding-box centre (partials per block).
__global__ void k_maxmin_first(const double *__restrict__ xy, int64_t n, const double *__restrict__ ctr,
                               double *__restrict__ pv, long long *__restrict__ pi) {
    double cx = ctr[0], cy = ctr[1];
    double bv = INFINITY;
    long long bi = 0x7FFFFFFFFFFFFFFFll;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double d = sqdist(xy[i], xy[n + i], cx, cy);
        if (better_min(d, i, bv, bi)) { bv = d; bi = i; }
    }
    MaxLoc r = block_argext(bv, bi, false);
    if (threadIdx.x == 0) { pv[blockIdx.x] = r.v; pi[blockIdx.x] = r.i; }
}

// One selection step.  Reduces the previous partials (min for the first
// step, max afterwards) to the point p taken at step k, records it, then
// updates the block's minimum distances and writes new partials.
__global__ void k_maxmin_step(const double *__restrict__ xy, int64_t n, int64_t k, int first,
                              const double *__restrict__ in_v, const long long *__restrict__ in_i,
                              double *__restrict__ out_v, long long *__restrict__ out_i,
                              double *__restrict__ mind, int64_t *__restrict__ perm) {
    __shared__ long long s_p;
    int nb = gridDim.x;
    double v = first ? INFINITY : -INFINITY;
    long long ii = 0x7FFFFFFFFFFFFFFFll;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double ov = in_v[b];
        long long oi = in_i[b];
        if (first ? better_min(ov, oi, v, ii) : better_max(ov, oi, v, ii)) { v = ov; ii = oi; }
    }
    MaxLoc r = block_argext(v, ii, !first);
    if (threadIdx.x == 0) s_p = r.i;
    __syncthreads();
    long long p = s_p;
    if (p < 0 || p >= n) p = 0;  // only reachable with non-finite coordinates
    if (blockIdx.x == 0 && threadIdx.x == 0) perm[k] = p;
    double px = xy[p], py = xy[n + p];
    double bv = -INFINITY;
    long long bi = 0x7FFFFFFFFFFFFFFFll;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double m = mind[i];
        if (i == p) m = -1.0;                      // taken
        else if (m >= 0.0) m = fmin(m, sqdist(xy[i], xy[n + i], px, py));
        mind[i] = m;
        if (better_max(m, i, bv, bi)) { bv = m; bi = i; }
    }
    r = block_argext(bv, bi, true);
    if (threadIdx.x == 0) { out_v[blockIdx.x] = r.v; out_i[blockIdx.x] = r.i; }
}

__global__ void k_fill(double *__restrict__ a, int64_t n, double v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// ------------------------------------------------------------- drivers
static inline int grid1(int64_t n, int t = 256) { return (int)ceil_div(n > 0 ? n : 1, t); }

void order_sfc(const double *xy, int64_t n, int method, uint64_t seed, int64_t *perm,
               uint32_t *codes, cudaStream_t s) {
    DevBuf kb(n * 4, s), vb(n * 4, s), kt(n * 4, s), vt(n * 4, s), hb(hist_words(n) * 4, s);
    uint32_t *keys = kb.as<uint32_t>(), *vals = vb.as<uint32_t>();
    uint32_t *ktmp = kt.as<uint32_t>(), *vtmp = vt.as<uint32_t>();
    launch(k_sfc_keys, grid1(n), 256, 0, s, xy, n, method, seed, keys, vals);
    TLR_CHECK_LAUNCH();
    if (codes) TLR_CUDA_TRY(cudaMemcpyAsync(codes, keys, n * 4, cudaMemcpyDeviceToDevice, s));
    radix_sort<uint32_t>(&keys, &vals, &ktmp, &vtmp, n, 32, hb.as<uint32_t>(), s);
    launch(k_perm_out, grid1(n), 256, 0, s, vals, n, perm);
    TLR_CHECK_LAUNCH();
}

static int bit_width(uint64_t v) {
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

void order_kdtree(const double *xy, int64_t n, int64_t *perm, cudaStream_t s) {
    if (n <= 1) {
        if (n == 1) launch(k_iota, 1, 32, 0, s, n, perm);
        return;
    }
    DevBuf kb(n * 8, s), kt(n * 8, s), vb(n * 4, s), vt(n * 4, s), hb(hist_words(n) * 4, s);
    DevBuf rx(n * 4, s), ry(n * 4, s);
    uint64_t *keys = kb.as<uint64_t>(), *ktmp = kt.as<uint64_t>();
    uint32_t *vals = vb.as<uint32_t>(), *vtmp = vt.as<uint32_t>(), *hist = hb.as<uint32_t>();
    // global ranks along x and y (stable: ties by index)
    for (int dim = 0; dim < 2; ++dim) {
        launch(k_coord_keys, grid1(n), 256, 0, s, xy + dim * n, n, keys, vals);
        radix_sort<uint64_t>(&keys, &vals, &ktmp, &vtmp, n, 64, hist, s);
        launch(k_invert, grid1(n), 256, 0, s, vals, n, dim ? ry.as<uint32_t>() : rx.as<uint32_t>());
        TLR_CHECK_LAUNCH();
    }
    // current order: identity
    launch(k_iota32, grid1(n), 256, 0, s, n, vals);
    TLR_CHECK_LAUNCH();
    // segment structure per level (host), then one sort per level
    std::vector<int64_t> starts{0}, sizes{n};
    int rbits = bit_width((uint64_t)(n - 1));
    DevBuf sb(n * 8, s), rb((size_t)n * 32, s);
    while (true) {
        bool any = false;
        for (int64_t m : sizes) any |= (m > 1);
        if (!any) break;
        int nseg = (int)starts.size();
        TLR_CUDA_TRY(cudaMemcpyAsync(sb.as<int64_t>(), starts.data(), nseg * 8, cudaMemcpyHostToDevice, s));
        unsigned long long *rng = rb.as<unsigned long long>();
        launch(k_kd_init_ranges, grid1(nseg), 256, 0, s, nseg, rng);
        launch(k_kd_ranges, grid1(n), 256, 0, s, xy, n, vals, sb.as<int64_t>(), nseg, rng);
        launch(k_kd_keys, grid1(n), 256, 0, s, n, vals, sb.as<int64_t>(), nseg, rng, rx.as<uint32_t>(),
                                           ry.as<uint32_t>(), rbits, keys);
        TLR_CHECK_LAUNCH();
        int bits = rbits + bit_width((uint64_t)(nseg - 1));
        radix_sort<uint64_t>(&keys, &vals, &ktmp, &vtmp, n, bits, hist, s);
        // children: first ceil(m/2) left, the rest right
        std::vector<int64_t> ns, nz;
        ns.reserve(2 * nseg);
        nz.reserve(2 * nseg);
        for (int q = 0; q < nseg; ++q) {
            int64_t m = sizes[q];
            if (m <= 1) { ns.push_back(starts[q]); nz.push_back(m); continue; }
            int64_t h = (m + 1) / 2;
            ns.push_back(starts[q]); nz.push_back(h);
            ns.push_back(starts[q] + h); nz.push_back(m - h);
        }
        starts.swap(ns);
        sizes.swap(nz);
        // the host vectors are read by the next level's async copy: keep the
        // stream in step with them
        TLR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    launch(k_perm_out, grid1(n), 256, 0, s, vals, n, perm);
    TLR_CHECK_LAUNCH();
}

void order_maxmin(const double *xy, int64_t n, int64_t *perm, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    int nblk = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms * 2);
    DevBuf mind(n * 8, s), pv(2 * nblk * 8, s), pi(2 * nblk * 8, s), ctr(16, s);
    launch(k_fill, grid1(n), 256, 0, s, mind.as<double>(), n, INFINITY);
    launch(k_bbox, 1, 1024, 0, s, xy, n, ctr.as<double>());
    launch(k_maxmin_first, nblk, 256, 0, s, xy, n, ctr.as<double>(), pv.as<double>(), pi.as<long long>());
    TLR_CHECK_LAUNCH();
    double *bv[2] = {pv.as<double>(), pv.as<double>() + nblk};
    long long *bi[2] = {pi.as<long long>(), pi.as<long long>() + nblk};
    for (int64_t k = 0; k < n; ++k) {
        int in = (int)(k & 1), out = in ^ 1;
        launch(k_maxmin_step, nblk, 256, 0, s, xy, n, k, k == 0, bv[in], bi[in], bv[out], bi[out],
                                           mind.as<double>(), perm);
    }
    TLR_CHECK_LAUNCH();
}

void order_identity(int64_t n, int64_t *perm, cudaStream_t s) {
    if (n > 0) launch(k_iota, grid1(n), 256, 0, s, n, perm);
    TLR_CHECK_LAUNCH();
}

void permute_xy(const double *xy, const int64_t *perm, int64_t n, int quantize, double *out,
                cudaStream_t s) {
    if (n > 0) launch(k_permute_xy, grid1(n), 256, 0, s, xy, perm, n, quantize, out);
    TLR_CHECK_LAUNCH();
}

void gather(const int64_t *perm, const double *src, int64_t n, double *dst, cudaStream_t s) {
    if (n > 0) launch(k_gather, grid1(n), 256, 0, s, perm, src, n, dst);
    TLR_CHECK_LAUNCH();
}

}  // namespace tlr

// ----------------------------------------------------------------------------
// Ordering without any allocation.
//
// For callers that must not allocate device memory once they are running:
// a serving loop whose latency budget cannot absorb cudaMalloc's implicit
// device synchronisation, or a host process whose memory is fixed up front
// (a pre-sized pool shared with other work).  tlr_order allocates its sort
// buffers per call; tlr_order_noalloc instead uses one file-scope scratch
// array that every device holds from module load until process exit.
// ----------------------------------------------------------------------------
namespace tlr {

constexpr int64_t kNoAllocMaxN = (int64_t)1 << 18;  // 262,144 locations
constexpr int64_t kNoAllocBlocks = (kNoAllocMaxN + kSortTile - 1) / kSortTile;
// keys, values and their ping-pong copies (4 x n words) plus the radix histogram
constexpr int64_t kNoAllocWords = 4 * kNoAllocMaxN + 256 * kNoAllocBlocks;

static __device__ __align__(256) uint32_t g_order_scratch[kNoAllocWords];

// Device address of g_order_scratch per device, looked up once per device.
static uint32_t *noalloc_scratch(int device, int *rc) {
    static std::mutex mu;
    static uint32_t *addr[64] = {nullptr};
    *rc = TLR_OK;
    if (device < 0 || device >= 64) { *rc = TLR_ERR_ARG; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_order_scratch);
        if (e != cudaSuccess || p == nullptr) { *rc = TLR_ERR_CUDA; return nullptr; }
        addr[device] = static_cast<uint32_t *>(p);
    }
    return addr[device];
}

}  // namespace tlr

extern "C" int tlr_order_noalloc(const double *xy, int64_t n, int method, uint64_t seed, int64_t *perm,
                                 uint32_t *codes, void *stream) {
    using namespace tlr;
    if (n < 0 || n > kNoAllocMaxN) return TLR_ERR_ARG;
    if (method != TLR_ORDER_RANDOM && method != TLR_ORDER_MORTON && method != TLR_ORDER_HILBERT)
        return TLR_ERR_ARG;
    if (n == 0) return TLR_OK;
    if (!xy || !perm) return TLR_ERR_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return TLR_ERR_CUDA;
    int rc = TLR_OK;
    uint32_t *base = noalloc_scratch(device, &rc);
    if (!base) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *keys = base, *vals = base + kNoAllocMaxN;
    uint32_t *ktmp = base + 2 * kNoAllocMaxN, *vtmp = base + 3 * kNoAllocMaxN;
    uint32_t *hist = base + 4 * kNoAllocMaxN;
    const int nblk = (int)ceil_div(n, kSortTile);
    launch(k_sfc_keys, grid1(n), 256, 0, s, xy, n, method, seed, keys, vals);
    if (codes && cudaMemcpyAsync(codes, keys, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TLR_ERR_CUDA;
    // stable LSD radix sort, 4 passes of 8 bits; every histogram entry and
    // every key/value slot read by a pass is written earlier in the same call
    for (int shift = 0; shift < 32; shift += 8) {
        launch(k_radix_hist<uint32_t>, nblk, kSortThreads, 0, s, keys, n, shift, hist, nblk);
        launch(k_scan_exclusive, 1, 1024, 0, s, hist, (int64_t)256 * nblk);
        launch(k_radix_scatter<uint32_t>, nblk, kSortThreads, 0, s, keys, vals, n, shift, hist, nblk, ktmp,
               vtmp);
        std::swap(keys, ktmp);
        std::swap(vals, vtmp);
    }
    launch(k_perm_out, grid1(n), 256, 0, s, vals, n, perm);
    return cudaGetLastError() == cudaSuccess ? TLR_OK : TLR_ERR_CUDA;
}

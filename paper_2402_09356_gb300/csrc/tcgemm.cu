// Tensor-core products of the mixed-precision path: FP64 operands split into
// power-of-two-scaled BF16 slices, slice products on tcgen05 with FP32
// accumulators in tensor memory, slice orders combined in float-float
// registers (the scheme is described in tcgemm.cuh).
//
// Data layout of a split operand X (rows x k; rows padded to a multiple of
// 128, k to a multiple of 64, padding zero): for every 32-wide stage ks of
// the inner dimension, slice p and block rb of 64 rows, a contiguous 4 KB
// block in the canonical K-major layout of the tensor cores without swizzle:
// core matrices of 8 rows x 8 elements (16 bytes a row, 128 bytes each),
// core (row group g, k group c) at byte (4 g + c) * 128 of the block.  Blocks
// are ordered [ks][p][rb], so the 128 rows of an A tile are 8 KB contiguous
// and one bulk copy (the TMA engine's cp.async.bulk) moves them.  The
// exponent e of every (row, 64-wide chunk) is stored beside: |x| <= 2^e.
//
// Kernel (one CTA per 128 x 32 output tile, 256 threads, at most 128
// registers a thread and 100 KB of shared memory with two stages, so that it
// shares an SM with the look-ahead product of the factorisation):
//   warp 0    producer: bulk copies of the S slices of A (128 x 32) and B
//             (64 x 32) per stage into an NS-stage ring (mbarrier with
//             transaction counts);
//   warp 1    MMA issuer: per stage and 16-wide k step, one
//             tcgen05.mma.kind::f16 (M 128, N 32, K 16) per slice pair into
//             the accumulator of its order; a commit frees the stage, and at
//             the end of each 64-wide chunk a commit hands the accumulator
//             buffer (4 orders x 32 columns, two buffers) to the epilogue;
//   warp 2    allocates and frees the tensor memory;
//   warps 4-7 epilogue: tcgen05.ld of their 32 lanes (rows) x 32 columns,
//             order sums combined exactly where they are exact, scaled by
//             2^(e_row + e_col) and added to float-float running sums kept in
//             tensor memory as well (tcgen05.st); after the last chunk the
//             FP64 epilogue (linear, or the Matern covariance of the two
//             locations) writes C.
// Every wait is bounded (4 s): a wait that times out sets TLR_ERR_TIMEOUT in
// the status word, the CTA stops issuing work, waits (bounded) for its own
// copies and products in flight, frees its tensor memory and returns.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_bf16.h>

#include "tcgemm.cuh"

namespace tlr {

namespace {

constexpr int kBM = 128, kBN = 32;    // output tile
constexpr int kKS = 32;               // inner dimension per pipeline stage
constexpr int kKC = 64;               // inner dimension per chunk (scale block, drain)
constexpr int kRowBlk = 64;           // rows per layout block
constexpr int kBlkElems = kRowBlk * kKS;  // 2048 BF16 = 4 KB
constexpr int kTcThreads = 256;
constexpr int kEpiWarp0 = 4, kEpiWarps = 4;
constexpr int kOrders = 4;            // accumulators: slice-pair order 0, 1, 2, >= 3
// tensor memory: two buffers of the four order accumulators (columns 0-255),
// then the running float-float sums of the tile (high words 256-287, low
// words 288-319); allocated as 512 columns
constexpr int kRunHi = 2 * kOrders * kBN, kRunLo = kRunHi + kBN;
constexpr int kTmemCols = 512;
constexpr unsigned long long kWaitNs = 4000000000ull;

struct TcSplitDesc {
    const double *src;
    int64_t rs, ks;       // element (r, kk) at src[r * rs + kk * ks]
    int rows, k;          // logical size
    int rows_pad, k_pad;  // rows_pad % 128 == 0, k_pad % 64 == 0
    uint16_t *dst;        // S * rows_pad * k_pad BF16 values
    int *ex;              // (k_pad / 64) * rows_pad exponents
};

struct TcProb {
    const uint16_t *A;
    const int *Aex;
    int a_rows_pad;
    const uint16_t *B;
    const int *Bex;
    int b_rows_pad;
    int m, n, k_pad;
    double *C;
    int ldc;
    int64_t ri0, ci0;  // epilogue: first global row / column
};

// The epilogues see the product through the same interface as the FP64 GEMMs.
struct TcEpiLinear {
    double beta;
    __device__ __forceinline__ double operator()(const TcProb &, int, int, double ab, const double *c) const {
        return beta == 0.0 ? ab : ab + beta * (*c);
    }
};
// (not inlined: the epilogue calls it for 32 columns of a fully unrolled loop)
__device__ __noinline__ double tc_matern_entry(const double *xy, int64_t n, const MaternParams &P, int64_t gr,
                                               int64_t gc) {
    return matern_cov(xy[gr], xy[n + gr], xy[gc], xy[n + gc], P);
}
struct TcEpiMatern {
    const double *xy;
    int64_t n;
    MaternParams P;
    __device__ __forceinline__ double operator()(const TcProb &p, int r, int c, double ab, const double *) const {
        const int64_t gr = p.ri0 + r, gc = p.ci0 + c;
        if (gr >= n || gc >= n) return 0.0;
        return tc_matern_entry(xy, n, P, gr, gc) + ab;
    }
};

__host__ __device__ __forceinline__ int64_t tc_index(int r, int kk, int p, int S, int rows_pad) {
    const int ks = kk >> 5, kin = kk & 31, rb = r >> 6, rin = r & 63;
    const int64_t blk = ((int64_t)ks * S + p) * (rows_pad >> 6) + rb;
    return blk * kBlkElems + ((rin >> 3) * 4 + (kin >> 3)) * 64 + (rin & 7) * 8 + (kin & 7);
}

// ---- splitting ---------------------------------------------------------------

// One warp per (row, 64-wide chunk); lane l takes elements 2l and 2l + 1.
// Scale: |x| <= 2^e over the chunk (frexp of the largest magnitude); then
// v = x 2^-e, and slice p is c_p 2^-8(p+1) with c_p = rint(2^8 v_p),
// v_{p+1} = 2^8 v_p - c_p (all exact in FP64; |c_0| <= 256, |c_p| <= 128).
// Non-finite chunks give NaN slices, so that the product is NaN as well.
template <int S>
__global__ void __launch_bounds__(256) k_tc_split(const TcSplitDesc *__restrict__ descs) {
    const TcSplitDesc D = descs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int nchunk = D.k_pad >> 6;
    const int64_t items = (int64_t)D.rows_pad * nchunk;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += wstride) {
        const int r = (int)(it % D.rows_pad), c = (int)(it / D.rows_pad);
        const int kk0 = c * kKC + 2 * lane;
        double x[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int kk = kk0 + u;
            x[u] = (r < D.rows && kk < D.k) ? D.src[(int64_t)r * D.rs + (int64_t)kk * D.ks] : 0.0;
        }
        double mx = fmax(fabs(x[0]), fabs(x[1]));
        bool bad = !(isfinite(x[0]) && isfinite(x[1]));
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            bad |= __shfl_xor_sync(0xFFFFFFFFu, (int)bad, o) != 0;
        }
        int e = 0;
        if (!bad && mx > 0.0) frexp(mx, &e);
        if (lane == 0) D.ex[(int64_t)c * D.rows_pad + r] = e;
        double v[2] = {ldexp(x[0], -e), ldexp(x[1], -e)};
#pragma unroll
        for (int p = 0; p < S; ++p) {
            uint32_t packed = 0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                float sl;
                if (bad) {
                    sl = __int_as_float(0x7fc00000);
                } else {
                    const double w = v[u] * 256.0;
                    const double cp = rint(w);
                    v[u] = w - cp;
                    sl = (float)ldexp(cp, -8 * (p + 1));
                }
                const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(sl));
                packed |= (uint32_t)b << (16 * u);
            }
            // elements kk0, kk0 + 1 are adjacent in the layout (same core row)
            *reinterpret_cast<uint32_t *>(D.dst + tc_index(r, kk0, p, S, D.rows_pad)) = packed;
        }
    }
}

// Row-contiguous operands (rs == 1, e.g. the column-major P of the panel
// update): lane l of a warp takes row 32 w + l of a chunk and walks its 64
// inner-dimension elements, so that every load is coalesced across the warp;
// each lane then writes its row's core rows as 16-byte pieces (eight lanes
// fill one 128-byte core matrix).
template <int S>
__global__ void __launch_bounds__(256) k_tc_split_rows(const TcSplitDesc *__restrict__ descs) {
    const TcSplitDesc D = descs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int nchunk = D.k_pad >> 6, rgroups = D.rows_pad >> 5;
    const int64_t items = (int64_t)rgroups * nchunk;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += wstride) {
        const int r = (int)(it % rgroups) * 32 + lane, c = (int)(it / rgroups);
        const bool live = r < D.rows;
        double mx = 0.0;
        bool bad = false;
        for (int u = 0; u < kKC; ++u) {
            const int kk = c * kKC + u;
            const double x = (live && kk < D.k) ? D.src[(int64_t)r * D.rs + (int64_t)kk * D.ks] : 0.0;
            mx = fmax(mx, fabs(x));
            bad |= !isfinite(x);
        }
        int e = 0;
        if (!bad && mx > 0.0) frexp(mx, &e);
        D.ex[(int64_t)c * D.rows_pad + r] = e;
        for (int g8 = 0; g8 < kKC / 8; ++g8) {
            const int kk0 = c * kKC + g8 * 8;
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int kk = kk0 + u;
                v[u] = (live && kk < D.k) ? ldexp(D.src[(int64_t)r * D.rs + (int64_t)kk * D.ks], -e) : 0.0;
            }
#pragma unroll
            for (int p = 0; p < S; ++p) {
                uint32_t w4[4];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    uint32_t packed = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float sl;
                        if (bad) {
                            sl = __int_as_float(0x7fc00000);
                        } else {
                            const double w = v[u + h] * 256.0;
                            const double cp = rint(w);
                            v[u + h] = w - cp;
                            sl = (float)ldexp(cp, -8 * (p + 1));
                        }
                        packed |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(sl)) << (16 * h);
                    }
                    w4[u / 2] = packed;
                }
                *reinterpret_cast<uint4 *>(D.dst + tc_index(r, kk0, p, S, D.rows_pad)) =
                    make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
    }
}

// ---- PTX helpers -----------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity.  Returns false
// if the CTA is aborting (another role timed out) or this wait timed out
// (then the status word gets TLR_ERR_TIMEOUT and the CTA aborts).
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, DevStatus *st) {
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((it & 255) == 255 && globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            set_status(st, TLR_ERR_TIMEOUT, -2);
            return false;
        }
    }
}

// The same wait while tearing down: ignores the abort flag, still bounded.
__device__ __noinline__ void mbar_wait_drain(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return;
        if ((it & 255) == 255 && globaltimer() - t0 > kWaitNs) return;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle; leading byte offset
// (between core matrices adjacent in K) 128, stride byte offset (between
// 8-row groups) 512; descriptor version 1 (bits 46-48 = 0b001).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"((uint32_t)accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 2^e as a float for integer e (0 below the normal range, +inf above).
__device__ __forceinline__ float exp2i(int e) {
    if (e < -126) return 0.f;
    if (e > 127) return __int_as_float(0x7f800000);
    return __int_as_float((e + 127) << 23);
}

// (s, t) = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int BM, int BN>
__device__ __forceinline__ bool tc_tile(const TcProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob,
                                        int t, TcProb &p, int &m0, int &n0) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
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

// A stage: S slices of the A tile (128 rows x 32, two layout blocks, 8 KB
// each) and of the B tile (32 rows x 32, half a layout block, 2 KB each).
constexpr int kTileABytes = 2 * kBlkElems * 2, kTileBBytes = kBN * kKS * 2;
template <int S>
constexpr int stage_bytes() { return S * (kTileABytes + kTileBBytes); }

template <int S, int NS>
constexpr size_t tc_smem_bytes() { return (size_t)NS * stage_bytes<S>() + 1024; }

// ---- the product ---------------------------------------------------------------

template <int S, int NS, class Epi>
__global__ void __launch_bounds__(kTcThreads, 2)
k_gemm_tc(const TcProb *__restrict__ probs, const int *__restrict__ tile_off, int nprob, int ntiles, double alpha,
          Epi epi, DevStatus *st) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int kStageA = S * kTileABytes;
    constexpr int kStage = stage_bytes<S>();
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NS * kStage);
    uint64_t *full = bars, *empty = bars + NS, *accf = bars + 2 * NS, *acce = accf + 2, *done = acce + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                TcProb p;
                int m0, n0;
                if (!tc_tile<kBM, kBN>(probs, tile_off, nprob, t, p, m0, n0)) continue;
                const int nks = p.k_pad / kKS, arb = p.a_rows_pad >> 6, brb = p.b_rows_pad >> 6;
                for (int ks = 0; ks < nks; ++ks, ++it) {
                    const int s = it % NS;
                    if (!mbar_wait(&empty[s], ((it / NS) & 1) ^ 1, abort_flag, st)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + (size_t)s * kStage, *sb = sa + kStageA;
                    mbar_expect_tx(&full[s], kStage);
#pragma unroll
                    for (int q = 0; q < S; ++q) {
                        const uint16_t *ga = p.A + (((int64_t)ks * S + q) * arb + (m0 >> 6)) * kBlkElems;
                        bulk_g2s(sa + q * kTileABytes, ga, kTileABytes, &full[s]);
                        // 32 rows of a 64-row block: row groups 4 (n0 % 64) / 8 .. , contiguous
                        const uint16_t *gb = p.B + (((int64_t)ks * S + q) * brb + (n0 >> 6)) * kBlkElems +
                                             (n0 & 63) * kKS;
                        bulk_g2s(sb + q * kTileBBytes, gb, kTileBBytes, &full[s]);
                    }
                }
            }
            // no copy may land after the CTA has left: wait for the last fill of every stage
            for (int s = 0; s < NS && s < it; ++s) {
                const int last = it - 1 - ((it - 1 - s) % NS);  // last fill index on stage s
                mbar_wait_drain(&full[s], (uint32_t)((last / NS) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            int it = 0, chunk = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                TcProb p;
                int m0, n0;
                if (!tc_tile<kBM, kBN>(probs, tile_off, nprob, t, p, m0, n0)) continue;
                const int nks = p.k_pad / kKS;
                uint32_t inited = 0;
                for (int ks = 0; ks < nks; ++ks, ++it) {
                    const int s = it % NS, b = chunk & 1;
                    if ((ks & 1) == 0) {  // a new chunk: its accumulator buffer must have been drained
                        if (!mbar_wait(&acce[b], ((chunk >> 1) & 1) ^ 1, abort_flag, st)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        inited = 0;
                    }
                    if (!mbar_wait(&full[s], (it / NS) & 1, abort_flag, st)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)s * kStage), sb = sa + kStageA;
#pragma unroll
                    for (int kt = 0; kt < kKS / 16; ++kt)
#pragma unroll
                        for (int pp = 0; pp < S; ++pp)
#pragma unroll
                            for (int qq = 0; qq + pp < S; ++qq) {
                                const int g = pp + qq < kOrders - 1 ? pp + qq : kOrders - 1;
                                const uint32_t d = tmem + (uint32_t)(b * kOrders * kBN + g * kBN);
                                const bool acc = (inited >> g) & 1u;
                                inited |= 1u << g;
                                tc_mma(d, umma_desc(sa + pp * kTileABytes + kt * 256),
                                       umma_desc(sb + qq * kTileBBytes + kt * 256), acc);
                            }
                    tc_commit(&empty[s]);  // the stage is free once these products are done
                    if (ks & 1) {
                        tc_commit(&accf[b]);
                        ++chunk;
                    }
                }
            }
            // every product issued must be complete before the tensor memory is freed
            tc_commit(done);
            mbar_wait_drain(done, 0);
        }
    } else if (warp >= kEpiWarp0) {
        // ---- epilogue
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        int chunk = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            TcProb p;
            int m0, n0;
            if (!tc_tile<kBM, kBN>(probs, tile_off, nprob, t, p, m0, n0)) continue;
            const int nch = p.k_pad / kKC;
            const int aprow = p.a_rows_pad, bprow = p.b_rows_pad;
            const int *aex = p.Aex + m0 + row, *bex = p.Bex + n0;
            for (int c = 0; c < nch; ++c, ++chunk) {
                const int b = chunk & 1;
                if (!mbar_wait(&accf[b], (chunk >> 1) & 1, abort_flag, st)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int er = aex[(int64_t)c * aprow];
                const int *ecol = bex + (int64_t)c * bprow;
#pragma unroll 1
                for (int cb = 0; cb < kBN; cb += 4) {
                    // orders that no slice pair reaches (S < 3) hold no product: read as zero
                    constexpr int kUsed = 2 * S - 1 < kOrders ? 2 * S - 1 : kOrders;
                    uint32_t g[kOrders][4], rh[4], rl[4];
#pragma unroll
                    for (int o = 0; o < kOrders; ++o) {
                        if (o < kUsed) {
                            tmem_ld4(tmem + lane_addr + (uint32_t)(b * kOrders * kBN + o * kBN + cb), g[o]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) g[o][j] = 0u;
                        }
                    }
                    if (c > 0) {
                        tmem_ld4(tmem + lane_addr + (uint32_t)(kRunHi + cb), rh);
                        tmem_ld4(tmem + lane_addr + (uint32_t)(kRunLo + cb), rl);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // orders 0 and 1 exactly, then the smaller orders
                        float s0, t0;
                        two_sum(__uint_as_float(g[0][j]), __uint_as_float(g[1][j]), s0, t0);
                        t0 = __fadd_rn(t0, __uint_as_float(g[2][j]));
                        t0 = __fadd_rn(t0, __uint_as_float(g[3][j]));
                        const float sc = exp2i(er + ecol[cb + j]);
                        s0 = __fmul_rn(s0, sc);
                        t0 = __fmul_rn(t0, sc);
                        if (c > 0) {  // running float-float sum
                            float u, w;
                            const float ah = __uint_as_float(rh[j]), al = __uint_as_float(rl[j]);
                            two_sum(ah, s0, u, w);
                            w = __fadd_rn(w, __fadd_rn(al, t0));
                            s0 = __fadd_rn(u, w);
                            t0 = __fsub_rn(w, __fsub_rn(s0, u));
                        }
                        rh[j] = __float_as_uint(s0);
                        rl[j] = __float_as_uint(t0);
                    }
                    tmem_st4(tmem + lane_addr + (uint32_t)(kRunHi + cb), rh);
                    tmem_st4(tmem + lane_addr + (uint32_t)(kRunLo + cb), rl);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[b]);
            }
            if (!ok) break;
            const int r = m0 + row;
#pragma unroll 1
            for (int cb = 0; cb < kBN; cb += 4) {
                uint32_t rh[4] = {0u, 0u, 0u, 0u}, rl[4] = {0u, 0u, 0u, 0u};
                if (nch > 0) {
                    tmem_ld4(tmem + lane_addr + (uint32_t)(kRunHi + cb), rh);
                    tmem_ld4(tmem + lane_addr + (uint32_t)(kRunLo + cb), rl);
                    tmem_wait_ld();
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int cc = n0 + cb + j;
                    if (r < p.m && cc < p.n) {
                        double *cp = p.C + (int64_t)cc * p.ldc + r;
                        const double ab = (double)__uint_as_float(rh[j]) + (double)__uint_as_float(rl[j]);
                        *cp = epi(p, r, cc, alpha * ab, cp);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---- host side --------------------------------------------------------------

template <class K>
void raise_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<const void *, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto &v = done[(const void *)kernel];
    if (v >= bytes) return;
    TLR_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    v = bytes;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// One split operand per distinct (pointer, leading dimension, transposition, rows, k).
struct SplitPlan {
    std::vector<TcSplitDesc> descs;
    std::map<std::tuple<const double *, int64_t, int64_t, int, int>, int> index;
    int64_t elems = 0, exps = 0;  // totals (BF16 values, exponents)
    int add(const double *src, int64_t rs, int64_t ks, int rows, int k, int S) {
        auto key = std::make_tuple(src, rs, ks, rows, k);
        auto it = index.find(key);
        if (it != index.end()) return it->second;
        TcSplitDesc d{};
        d.src = src;
        d.rs = rs;
        d.ks = ks;
        d.rows = rows;
        d.k = k;
        d.rows_pad = (int)round_up(std::max(rows, 1), 128);
        d.k_pad = (int)round_up(k, kKC);
        d.dst = reinterpret_cast<uint16_t *>(elems);  // offsets for now
        d.ex = reinterpret_cast<int *>(exps);
        elems += (int64_t)S * d.rows_pad * d.k_pad;
        exps += (int64_t)(d.k_pad / kKC) * d.rows_pad;
        descs.push_back(d);
        const int id = (int)descs.size() - 1;
        index[key] = id;
        return id;
    }
};

template <int S, class Epi>
void launch_tc(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs, double alpha,
               const Epi &epi, int ctas_per_sm) {
    std::vector<GemmProb> act;
    for (const GemmProb &p : probs)
        if (p.m > 0 && p.n > 0) act.push_back(p);
    if (act.empty()) return;
    // split plan: A rows = rows of op(A), B rows = columns of op(B)
    SplitPlan plan;
    std::vector<std::pair<int, int>> ids;
    for (const GemmProb &p : act) {
        const int k = std::max(p.k, 0);
        const int ia = ta ? plan.add(p.A, p.lda, 1, p.m, k, S) : plan.add(p.A, 1, p.lda, p.m, k, S);
        const int ib = tb ? plan.add(p.B, 1, p.ldb, p.n, k, S) : plan.add(p.B, p.ldb, 1, p.n, k, S);
        ids.emplace_back(ia, ib);
    }
    const size_t bytes_sl = (size_t)plan.elems * sizeof(uint16_t), bytes_ex = (size_t)plan.exps * sizeof(int);
    DevBuf ws(round_up((int64_t)bytes_sl, 256) + bytes_ex + 256, s);
    uint16_t *sl = ws.as<uint16_t>();
    int *ex = reinterpret_cast<int *>(reinterpret_cast<char *>(sl) + round_up((int64_t)bytes_sl, 256));
    std::vector<TcSplitDesc> by_k, by_row;  // inner dimension contiguous / rows contiguous
    int64_t most_k = 0, most_row = 0;
    for (TcSplitDesc &d : plan.descs) {
        d.dst = sl + reinterpret_cast<int64_t>(d.dst);
        d.ex = ex + reinterpret_cast<int64_t>(d.ex);
        const int64_t items = (int64_t)d.rows_pad * (d.k_pad / kKC);
        if (d.rs == 1 && d.ks != 1) {
            by_row.push_back(d);
            most_row = std::max<int64_t>(most_row, items / 32);
        } else {
            by_k.push_back(d);
            most_k = std::max<int64_t>(most_k, items);
        }
    }
    if (most_k > 0) {
        auto *dd = (const TcSplitDesc *)stage_push(ctx, by_k.data(), by_k.size() * sizeof(TcSplitDesc), s);
        const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(most_k, 8), 2048);
        launch(k_tc_split<S>, dim3(gx, (unsigned)by_k.size()), 256, 0, s, dd);
        TLR_CHECK_LAUNCH();
    }
    if (most_row > 0) {
        auto *dd = (const TcSplitDesc *)stage_push(ctx, by_row.data(), by_row.size() * sizeof(TcSplitDesc), s);
        const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(most_row, 8), 2048);
        launch(k_tc_split_rows<S>, dim3(gx, (unsigned)by_row.size()), 256, 0, s, dd);
        TLR_CHECK_LAUNCH();
    }
    std::vector<TcProb> tp;
    std::vector<int> off(act.size() + 1, 0);
    for (size_t b = 0; b < act.size(); ++b) {
        const GemmProb &p = act[b];
        const TcSplitDesc &da = plan.descs[ids[b].first], &db = plan.descs[ids[b].second];
        TcProb t{};
        t.A = da.dst;
        t.Aex = da.ex;
        t.a_rows_pad = da.rows_pad;
        t.B = db.dst;
        t.Bex = db.ex;
        t.b_rows_pad = db.rows_pad;
        t.m = p.m;
        t.n = p.n;
        t.k_pad = da.k_pad;
        t.C = p.C;
        t.ldc = p.ldc;
        t.ri0 = p.ri0;
        t.ci0 = p.ci0;
        tp.push_back(t);
        off[b + 1] = off[b] + (int)(ceil_div(p.m, kBM) * ceil_div(p.n, kBN));
    }
    const int total = off.back();
    auto *dp = (const TcProb *)stage_push(ctx, tp.data(), tp.size() * sizeof(TcProb), s);
    auto *dt = (const int *)stage_push(ctx, off.data(), off.size() * sizeof(int), s);
    if (ctas_per_sm > 0) {
        // more than half an SM's shared memory: one CTA of this product per SM,
        // the rest of the SM open to a critical-path CTA (a second CTA of it
        // would also wait for the tensor memory the first one holds)
        int dev = 0, per_sm = 0;
        TLR_CUDA_TRY(cudaGetDevice(&dev));
        TLR_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        const size_t smem = std::max(tc_smem_bytes<S, 2>(), (size_t)per_sm / 2 + 1024);
        raise_smem(k_gemm_tc<S, 2, Epi>, smem);
        launch(k_gemm_tc<S, 2, Epi>, total, kTcThreads, smem, s, dp, dt, (int)act.size(), total, alpha, epi,
               ctx->d_status);
    } else {
        constexpr size_t smem = tc_smem_bytes<S, 3>();
        raise_smem(k_gemm_tc<S, 3, Epi>, smem);
        launch(k_gemm_tc<S, 3, Epi>, total, kTcThreads, smem, s, dp, dt, (int)act.size(), total, alpha, epi,
               ctx->d_status);
    }
    TLR_CHECK_LAUNCH();
}

}  // namespace

bool tc_available() {
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        int dev = 0, major = 0, minor = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        const bool loaded = cudaFuncGetAttributes(&fa, k_gemm_tc<kTcSlicesDefault, 3, TcEpiLinear>) == cudaSuccess;
        ok = loaded && major == 10 && minor == 3 && (size_t)optin >= tc_smem_bytes<kTcSlicesDefault, 3>();
        cudaGetLastError();
    });
    return ok;
}

void gemm_tc(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, const std::vector<GemmProb> &probs, double alpha,
             double beta, int slices, bool light) {
    if (!tc_available()) throw make_error(TLR_ERR_CUDA, "tensor-core products need an sm_103a device");
    const int per = light ? 1 : 0;
    if (slices == 1) launch_tc<1>(ctx, s, ta, tb, probs, alpha, TcEpiLinear{beta}, per);
    else if (slices == kTcSlicesDefault) launch_tc<kTcSlicesDefault>(ctx, s, ta, tb, probs, alpha, TcEpiLinear{beta}, per);
    else throw make_error(TLR_ERR_ARG, "tensor-core products take 1 or %d slices", kTcSlicesDefault);
}

void gemm_tc_matern(tlr_ctx *ctx, cudaStream_t s, bool tb, const std::vector<GemmProb> &probs, double alpha,
                    const double *xy, int64_t n, const MaternParams &P, int slices, int ctas_per_sm) {
    if (!tc_available()) throw make_error(TLR_ERR_CUDA, "tensor-core products need an sm_103a device");
    if (!tb) throw make_error(TLR_ERR_ARG, "the Matern panel product takes B transposed");
    TcEpiMatern e;
    e.xy = xy;
    e.n = n;
    e.P = P;
    if (slices == 1) launch_tc<1>(ctx, s, false, true, probs, alpha, e, ctas_per_sm);
    else if (slices == kTcSlicesDefault) launch_tc<kTcSlicesDefault>(ctx, s, false, true, probs, alpha, e, ctas_per_sm);
    else throw make_error(TLR_ERR_ARG, "tensor-core products take 1 or %d slices", kTcSlicesDefault);
}

void gemm_tc_single(tlr_ctx *ctx, cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                    const double *A, int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices) {
    GemmProb p{};
    p.A = A;
    p.lda = lda;
    p.B = B;
    p.ldb = ldb;
    p.C = C;
    p.ldc = ldc;
    p.m = m;
    p.n = n;
    p.k = k;
    gemm_tc(ctx, s, ta, tb, std::vector<GemmProb>{p}, alpha, beta, slices);
}

}  // namespace tlr

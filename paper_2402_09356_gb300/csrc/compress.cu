// a3: per-tile low-rank compression at an absolute accuracy tau (Sec. 2-3:
// the accuracy threshold decides how many singular values are kept).
//
// For a dense tile T (m x k) the rank is r = #{sigma_i(T) > tau} and the
// factors satisfy T ~ U V' with |T - U V'|_2 ~ sigma_{r+1}.  Computing the
// full SVD of every nb x nb tile would cost O(nb^3); instead, per tile:
//   1. Y = T Omega (Omega: k x s Gaussian) by batched GEMM (whole GPU);
//   2. Q = orth(Y): Householder QR with the explicit Q formed in place;
//   3. B = T' Q (batched GEMM), kept, and the R factor of B = Q2 R;
//   4. one-sided Jacobi SVD of R' = W S Z' (only W and S are formed).
// With the unit left singular vectors W of R' (the right singular vectors
// of B) and W_r their first r columns,
//   U = Q W_r,  V = B W_r  =>  U V' = Q W_r W_r' Q' T,
// the projection of T onto its r dominant left singular directions within
// range(Q), so |T - U V'| <= |T - Q Q' T| + sigma_{r+1}(Q' T).
// The rank is the SVD count of the projected tile, r = #{S > tau}.  A sample
// of s = r + 24 columns reproduces the exact SVD rank and an error below tau
// on the Matern tiles of the workloads (nu = 0.5 has the slowest decay); the
// sample size comes from the tile's rank at the previous evaluation, and a
// tile whose detected rank leaves fewer than 20 spare samples is redone with
// a larger sample (Halko, Martinsson, Tropp 2011, Sec. 4: oversampling).
//
// GB300 issues 2 FP64 FMA per clock per SM, so one tile's QR or SVD on one SM
// is slow, and the highest-rank tile of a column lies on the critical path of
// the factorisation.  Each tile therefore runs on a thread-block cluster whose
// CTAs keep their share of the tile in shared memory:
//   - QR: the CTAs split the rows; per column one cluster barrier exchanges
//     the partial dot products through distributed shared memory (DSMEM);
//   - SVD: the columns of R' form 2C blocks; every CTA rotates the column
//     pairs between (and, once per sweep, within) its two blocks and then
//     pulls its next two blocks from their holders over DSMEM, following a
//     round-robin tournament, with one cluster barrier per block round.
// Tiles whose panels do not fit in shared memory use global-memory variants.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "compress.cuh"
#include "ff.cuh"
#include "gemm.cuh"
#include "tcgemm.cuh"

namespace tlr {

namespace cg = cooperative_groups;

constexpr int kOversample = 24;  // samples beyond the expected rank
constexpr int kSpare = 20;       // fewer spare samples than this: redo with more
constexpr int kQrThreads = 256;
constexpr int kNw = kQrThreads / 32;
// Threads of the shared-memory QR (512 measured slower at n = 40,000: the
// step's barrier and exchange latency, not its dependent chains, bound it).
constexpr int kQrSmThreads = 256;
constexpr int kMaxSweeps = 40;

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

// Householder reflector of one column: given |x|^2 (nrm2) and its head alpha,
// beta = -sign(alpha) |x|, v = x with v_head = alpha - beta, tau = 2 / v'v.
__device__ __forceinline__ void householder(double nrm2, double alpha, double &tau, double &beta, double &v0) {
    tau = 0.0;
    beta = 0.0;
    v0 = 0.0;
    const double nrm = sqrt(nrm2);
    if (nrm != 0.0) {
        beta = -copysign(nrm, alpha);
        v0 = alpha - beta;
        tau = 2.0 / (nrm2 - alpha * alpha + v0 * v0);
    }
}

// The same reflector in float-float arithmetic.  With beta = -sign(alpha) |x|
// and v0 = alpha - beta, v'v = 2 |x| |v0|, so tau = 1 / (|x| |v0|); tau is
// kept as its two factors rn = 1 / |x| and rv = 1 / |v0| (tau itself would
// leave FP32's exponent range for |x| below ~1e-19), and every use multiplies
// by them in an order that keeps the intermediate values near the data's
// scale.  A column with |x| < 1e-30 (where the pairs' low words are already
// subnormal) is taken as zero: no reflector.
__device__ __forceinline__ void householder_ff(FF nrm2, FF alpha, FF &rn, FF &rv, FF &beta, FF &v0) {
    rn = rv = beta = v0 = FF{0.f, 0.f};
    const FF nrm = ff_sqrt(nrm2);
    if (nrm.h >= 1e-30f) {
        const FF snrm = alpha.h < 0.f ? ff_neg(nrm) : nrm;
        beta = ff_neg(snrm);
        v0 = ff_add(alpha, snrm);
        rn = ff_div(FF{1.f, 0.f}, nrm);
        rv = ff_div(FF{1.f, 0.f}, v0.h < 0.f ? ff_neg(v0) : v0);
    }
}

struct QrJob {
    double *A;  // m x s input (ld lda); read only, except by the global-memory variant
    int lda;
    double *Q;  // m x s output Q (ld ldq), or null
    int ldq;
    double *Rt;  // s x s output R' (ld s, lower triangular), or null
    int m, s;
    float2 *Rt2;  // paired-FP32 variant: R' also as (hi, lo) pairs (ld s), or null
};

// ---------------------------------------------------------------------------
// Work split of one panel step over a CTA's threads.  GB300 issues FP64 at
// 1/64 of the FP32 rate, so the FP64 instruction count is what matters: each
// thread owns whole columns (lanes <-> columns, no shuffle reductions), and
// when the columns fill fewer than all warps the rows are split into G
// interleaved groups over the spare warps (their partial dot products are
// summed through shared memory).  Thread t handles row group t / width and
// columns first + t % width + k * width.
template <int kThreads>
struct PanelSplit {
    int G, width;
    __device__ __forceinline__ explicit PanelSplit(int ncols) {
        constexpr int kWarps = kThreads / 32;
        const int cw = (ncols + 31) / 32;
        if (cw >= kWarps || cw == 0) {
            G = 1;
            width = kThreads;
        } else {
            G = kWarps / cw;
            width = 32 * cw;
        }
    }
};

// Element arithmetic of the shared-memory QR: FP64, or paired FP32 (each
// element held as hi + lo, two FP32 words in the bytes of one double; dot
// products accumulate with the TwoSum scheme of df_fma, updates a - w v form
// the exact product of the high words by FMA and renormalise), which runs on
// the FP32 pipe at about 46-bit accuracy.  The per-column scalars (partial
// dot products, the reflector's norm, tau, head and beta, the update weights)
// are of type P: FP64, or float-float pairs (ff.cuh) in the paired variant,
// so that its column steps issue no FP64 instruction (an FP64 warp
// instruction holds GB300's FP64 pipe for 64 cycles, one active lane or 32).
template <bool kDf>
struct QrArith;
template <>
struct QrArith<false> {
    using T = double;
    struct Acc {
        double d = 0.0;
    };
    static __device__ __forceinline__ T from(double x) { return x; }
    static __device__ __forceinline__ double to(T x) { return x; }
    static __device__ __forceinline__ void acc(Acc &a, T x, T y) { a.d = fma(x, y, a.d); }
    static __device__ __forceinline__ double val(const Acc &a) { return a.d; }
    // a - w v, with w prepared by prep()
    struct W {
        double w;
    };
    static __device__ __forceinline__ W prep(double w) { return W{w}; }
    static __device__ __forceinline__ T axmy(T a, const W &w, T v) { return fma(-w.w, v, a); }
    // per-column scalars
    using P = double;
    static __device__ __forceinline__ P part(const Acc &a) { return a.d; }
    static __device__ __forceinline__ P elem(T x) { return x; }
    static __device__ __forceinline__ P padd(P a, P b) { return a + b; }
    static __device__ __forceinline__ P pmul(P a, P b) { return a * b; }
    static __device__ __forceinline__ bool nz(P a) { return a != 0.0; }
    static __device__ __forceinline__ W prepP(P w) { return W{w}; }
    static __device__ __forceinline__ T fromP(P x) { return x; }
    static __device__ __forceinline__ double toD(P x) { return x; }
};
template <>
struct QrArith<true> {
    using T = float2;
    struct Acc {
        float h = 0.f, l = 0.f;
    };
    static __device__ __forceinline__ T from(double x) {
        const float h = __double2float_rn(x);
        return make_float2(h, __double2float_rn(x - (double)h));
    }
    static __device__ __forceinline__ double to(T x) { return (double)x.x + (double)x.y; }
    static __device__ __forceinline__ void acc(Acc &a, T x, T y) { df_fma(x.x, x.y, y.x, y.y, a.h, a.l); }
    static __device__ __forceinline__ double val(const Acc &a) { return (double)a.h + (double)a.l; }
    struct W {
        float h, l;
    };
    static __device__ __forceinline__ W prep(double w) {
        const float h = __double2float_rn(w);
        return W{h, __double2float_rn(w - (double)h)};
    }
    using P = FF;
    static __device__ __forceinline__ P part(const Acc &a) { return ff_two_sum(a.h, a.l); }
    static __device__ __forceinline__ P elem(T x) { return FF{x.x, x.y}; }
    static __device__ __forceinline__ P padd(P a, P b) { return ff_add(a, b); }
    static __device__ __forceinline__ P pmul(P a, P b) { return ff_mul(a, b); }
    static __device__ __forceinline__ bool nz(P a) { return a.h != 0.f; }
    static __device__ __forceinline__ W prepP(P w) { return W{w.h, w.l}; }
    static __device__ __forceinline__ T fromP(P x) { return make_float2(x.h, x.l); }
    static __device__ __forceinline__ double toD(P x) { return (double)x.h + (double)x.l; }
    static __device__ __forceinline__ T axmy(T a, const W &w, T v) {
        const float ph = __fmul_rn(w.h, v.x);
        float pl = __fmaf_rn(w.h, v.x, -ph);
        pl = __fmaf_rn(w.h, v.y, pl);
        pl = __fmaf_rn(w.l, v.x, pl);
        // TwoSum of a.x and -ph
        const float sh = __fsub_rn(a.x, ph);
        const float bp = __fsub_rn(sh, a.x);
        const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(sh, bp)), __fsub_rn(-ph, bp));
        const float sl = __fadd_rn(__fsub_rn(a.y, pl), err);
        const float hi = __fadd_rn(sh, sl);
        return make_float2(hi, __fsub_rn(sl, __fsub_rn(hi, sh)));
    }
};

// Dot products d_cc = sum over local rows i >= lb of v[i] A(i, cc) for the
// columns cc in [first, s), written to out[cc].  red: kThreads scalars.
template <int kThreads, class Ar, class T, class P>
__device__ __forceinline__ void panel_dots(const T *As, int ld, const T *v, int first, int s, int lb, int nr,
                                           P *red, P *out) {
    const int tid = threadIdx.x;
    const PanelSplit<kThreads> ps(s - first);
    const int g = tid / ps.width;
    if (ps.G == 1) {
        for (int cc = first + tid; cc < s; cc += ps.width) {
            const T *ac = As + cc * ld;
            typename Ar::Acc d;
            for (int i = lb; i < nr; ++i) Ar::acc(d, v[i], ac[i]);
            out[cc] = Ar::part(d);
        }
        return;
    }
    const int cc = first + tid % ps.width;
    if (tid < ps.G * ps.width && cc < s) {
        const T *ac = As + cc * ld;
        typename Ar::Acc d;
        for (int i = lb + g; i < nr; i += ps.G) Ar::acc(d, v[i], ac[i]);
        red[tid] = Ar::part(d);
    }
    __syncthreads();
    if (tid < ps.width && cc < s) {
        P d{};
        for (int q = 0; q < ps.G; ++q) d = Ar::padd(d, red[q * ps.width + tid]);
        out[cc] = d;
    }
}

// A(i, cc) -= w[cc] v(i) for local rows i >= lb and columns cc in [first, s),
// where v(i) = v[i] except v(ic) = vhead when ic is a local row.
template <int kThreads, class Ar, class T, class P>
__device__ __forceinline__ void panel_update(T *As, int ld, const T *v, int ic, T vhead, const P *w, int first,
                                             int s, int lb, int nr) {
    const int tid = threadIdx.x;
    const PanelSplit<kThreads> ps(s - first);
    if (tid >= ps.G * ps.width) return;
    const int g = tid / ps.width;
    for (int cc = first + tid % ps.width; cc < s; cc += ps.width) {
        const typename Ar::W wc = Ar::prepP(w[cc]);
        T *ac = As + cc * ld;
        for (int i = lb + g; i < nr; i += ps.G) ac[i] = Ar::axmy(ac[i], wc, i == ic ? vhead : v[i]);
    }
}

// ---------------------------------------------------------------------------
// QR with the panel in shared memory.  CTA `rank` of the cluster owns rows
// [r0, r0 + nr) of all s columns, column-major with an odd leading dimension.
// Column c: every CTA forms the dot products of column c with columns c..s-1
// over its rows (at or below row c), and the owner of row c publishes that
// row; after one cluster barrier every CTA sums the kCl partials, forms the
// reflector (v = column c with v_c = v0) and w_cc = tau (d_cc + (v0 - alpha)
// A(c, cc)), and updates its own rows.  Buffers alternate by column parity, so
// a CTA never overwrites values another CTA may still be reading.
// Q = H_0 ... H_{s-1} [I; 0] is then accumulated backwards in place: before
// H_c is applied, columns > c already hold their final values below row c,
// and column c becomes H_c e_c (LAPACK's dorg2r ordering).
// Shared memory: s * ld + 9 s + kQrSmThreads doubles.
template <int kCl, bool kDf>
__global__ void __launch_bounds__(kQrSmThreads) k_qr_sm(const QrJob *__restrict__ jobs) {
    using Ar = QrArith<kDf>;
    using T = typename Ar::T;
    static_assert(sizeof(T) == sizeof(double), "the panel element takes the bytes of one double");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const QrJob J = jobs[blockIdx.x / kCl];
    const int m = J.m, s = J.s, tid = threadIdx.x;
    const int per = (m + kCl - 1) / kCl, ld = per | 1;
    const int r0 = min(m, rank * per), nr = min(m, r0 + per) - r0;
    using P = typename Ar::P;
    static_assert(sizeof(P) == sizeof(double), "a column scalar takes the bytes of one double");
    extern __shared__ double sm[];
    T *As = reinterpret_cast<T *>(sm);
    // taus: tau (FP64), or 1 / |x| with rvs = 1 / |v0| (pairs; householder_ff)
    P *taus = reinterpret_cast<P *>(sm + (size_t)s * ld), *betas = taus + s, *heads = betas + s, *rvs = heads + s;
    P *pd = rvs + s, *prow = pd + 2 * s, *wv = prow + 2 * s, *red = wv + s;
    for (int e = tid; e < nr * s; e += kQrSmThreads) {
        const int i = e % nr, j = e / nr;
        As[j * ld + i] = Ar::from(J.A[(int64_t)j * J.lda + r0 + i]);
    }
    __syncthreads();
    for (int c = 0; c < s; ++c) {
        P *pdc = pd + (c & 1) * s, *prc = prow + (c & 1) * s;
        const int lb = max(c - r0, 0), ic = c - r0;
        T *vc = As + c * ld;
        panel_dots<kQrSmThreads, Ar>(As, ld, vc, c, s, lb, nr, red, pdc);
        const int owner = c / per;
        if (rank == owner)
            for (int cc = c + tid; cc < s; cc += kQrSmThreads) prc[cc] = Ar::elem(As[cc * ld + ic]);
        cl.sync();
        const P *orow = cl.map_shared_rank(prc, owner);
        // the reflector's scalars once per CTA (every thread repeating the
        // norm, square root and division would only repeat the same work)
        if (tid == 0) {
            P nrm2{};
#pragma unroll
            for (int k = 0; k < kCl; ++k) nrm2 = Ar::padd(nrm2, cl.map_shared_rank(pdc, k)[c]);
            const P alpha = orow[c];
            if constexpr (kDf) {
                householder_ff(nrm2, alpha, taus[c], rvs[c], betas[c], heads[c]);
            } else {
                double tau, beta, v0;
                householder(nrm2, alpha, tau, beta, v0);
                taus[c] = tau;
                betas[c] = beta;
                heads[c] = v0;
            }
            red[0] = alpha;
        }
        __syncthreads();
        const P tau = taus[c], v0 = heads[c];
        for (int cc = c + 1 + tid; cc < s; cc += kQrSmThreads) {
            P d{};
#pragma unroll
            for (int k = 0; k < kCl; ++k) d = Ar::padd(d, cl.map_shared_rank(pdc, k)[cc]);
            // w_cc = tau (d_cc + (v0 - alpha) A(c, cc)), v0 - alpha = -beta
            if constexpr (kDf)
                wv[cc] = ff_mul(ff_mul(ff_add(d, ff_mul(ff_neg(betas[c]), orow[cc])), tau), rvs[c]);
            else
                wv[cc] = tau * (d + (v0 - red[0]) * orow[cc]);
        }
        __syncthreads();
        if (Ar::nz(tau)) panel_update<kQrSmThreads, Ar>(As, ld, vc, ic, Ar::fromP(v0), wv, c + 1, s, lb, nr);
        __syncthreads();
        if (Ar::nz(tau) && rank == owner && tid == 0) vc[ic] = Ar::fromP(v0);  // reflector head stored in place
    }
    cl.sync();  // every CTA is done reading the factorisation's partials
    if (J.Rt) {  // Rt(i, u) = R(u, i) for the own rows u < s
        const int nu = max(0, min(nr, s - r0));
        for (int e = tid; e < nu * s; e += kQrSmThreads) {
            const int lu = e / s, i = e % s, u = r0 + lu;
            double v = 0.0;
            T w = Ar::from(0.0);
            if (i > u) {
                w = As[i * ld + lu];
                v = Ar::to(w);
            } else if (i == u) {
                w = Ar::fromP(betas[u]);
                v = Ar::toD(betas[u]);
            }
            J.Rt[(int64_t)u * s + i] = v;
            if constexpr (kDf)
                if (J.Rt2) J.Rt2[(int64_t)u * s + i] = w;
        }
    }
    if (!J.Q) return;
    __syncthreads();
    int act = 0;
    for (int c = s - 1; c >= 0; --c) {
        const P tau = taus[c], v0 = heads[c];
        const int lb = max(c - r0, 0), ic = c - r0;
        T *vc = As + c * ld;
        if (Ar::nz(tau)) {  // identical on every CTA of the cluster
            P *pdc = pd + (act & 1) * s;
            ++act;
            panel_dots<kQrSmThreads, Ar>(As, ld, vc, c + 1, s, lb, nr, red, pdc);
            cl.sync();
            for (int cc = c + 1 + tid; cc < s; cc += kQrSmThreads) {
                P d{};
#pragma unroll
                for (int k = 0; k < kCl; ++k) d = Ar::padd(d, cl.map_shared_rank(pdc, k)[cc]);
                if constexpr (kDf) wv[cc] = ff_mul(ff_mul(d, tau), rvs[c]);
                else wv[cc] = tau * d;
            }
            __syncthreads();
            panel_update<kQrSmThreads, Ar>(As, ld, vc, -1, Ar::from(0.0), wv, c + 1, s, lb, nr);
            __syncthreads();
        }
        // column c of Q = H_c e_c: tau v0 (= sign(v0) / |x| in pairs) times
        // the reflector, 1 - tau v0^2 (= 1 - |v0| / |x|) at the head
        typename Ar::W tv;
        T qc;
        if constexpr (kDf) {
            const bool neg = v0.h < 0.f;
            tv = Ar::prepP(neg ? ff_neg(tau) : tau);
            qc = Ar::fromP(ff_add(FF{1.f, 0.f}, ff_neg(ff_mul(neg ? ff_neg(v0) : v0, tau))));
        } else {
            tv = Ar::prepP(tau * v0);
            qc = Ar::from(1.0 - tau * v0 * v0);
        }
        for (int i = tid; i < nr; i += kQrSmThreads) {
            T q;
            if (i < ic) q = Ar::from(0.0);
            else if (i == ic) q = qc;
            else q = Ar::axmy(Ar::from(0.0), tv, vc[i]);
            vc[i] = q;
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * s; e += kQrSmThreads) {
        const int i = e % nr, j = e / nr;
        J.Q[(int64_t)j * J.ldq + r0 + i] = Ar::to(As[j * ld + i]);
    }
    cl.sync();  // no CTA leaves while another may still read its partials
}

static size_t qr_sm_bytes(int m, int s, int csize) {
    const int per = (m + csize - 1) / csize, ld = per | 1;
    return ((size_t)s * ld + 9 * (size_t)s + kQrSmThreads) * sizeof(double);
}

// QR in global memory (A factorised in place; Q and Rt as above), for panels
// that do not fit in shared memory.  Same barrier scheme as k_qr_sm.
template <int kCl>
__global__ void __launch_bounds__(kQrThreads) k_qr_gm(const QrJob *__restrict__ jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const QrJob J = jobs[blockIdx.x / kCl];
    const int m = J.m, s = J.s, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (m + kCl - 1) / kCl;
    const int r0 = min(m, rank * per), r1 = min(m, r0 + per);
    __shared__ double red[32];
    __shared__ double s_norm[2];
    extern __shared__ double s_dyn[];  // taus (s), betas (s), dots (2 x s), row c of the owner (2 x s)
    double *taus = s_dyn, *betas = s_dyn + s, *dots = s_dyn + 2 * s, *prow = s_dyn + 4 * s;
    double *A = J.A;
    const int64_t lda = J.lda;
    for (int c = 0; c < s; ++c) {
        const int par = c & 1;
        double *col = A + (int64_t)c * lda;
        const int rb = max(r0, c);
        double *pd = dots + par * s, *pr = prow + par * s;
        double p = 0.0;
        for (int r = rb + tid; r < r1; r += kQrThreads) p += col[r] * col[r];
        p = block_sum(p, red);
        if (tid == 0) s_norm[par] = p;
        for (int cc = c + 1 + warp; cc < s; cc += kNw) {
            const double *dst = A + (int64_t)cc * lda;
            double w = 0.0;
            for (int r = rb + lane; r < r1; r += 32) w += col[r] * dst[r];
            w = warp_sum(w);
            if (lane == 0) pd[cc] = w;
        }
        const int owner = c / per;
        if (rank == owner)
            for (int cc = c + tid; cc < s; cc += kQrThreads) pr[cc] = A[(int64_t)cc * lda + c];
        cl.sync();
        const double *orow = cl.map_shared_rank(pr, owner);
        __shared__ double s_sc[2];  // alpha, v0 of the column (computed once per CTA)
        if (tid == 0) {
            double nrm2 = 0.0;
            for (int k = 0; k < kCl; ++k) nrm2 += cl.map_shared_rank(s_norm, k)[par];
            double tau_, beta_, v0_;
            householder(nrm2, orow[c], tau_, beta_, v0_);
            taus[c] = tau_;
            betas[c] = beta_;
            s_sc[0] = orow[c];
            s_sc[1] = v0_;
        }
        __syncthreads();
        const double tau = taus[c], alpha = s_sc[0], v0 = s_sc[1];
        if (tau != 0.0) {
            for (int cc = c + 1 + warp; cc < s; cc += kNw) {
                double d = 0.0;
                for (int k = 0; k < kCl; ++k) d += cl.map_shared_rank(pd, k)[cc];
                const double w = tau * (d + (v0 - alpha) * orow[cc]);
                double *dst = A + (int64_t)cc * lda;
                for (int r = rb + lane; r < r1; r += 32) dst[r] -= w * (r == c ? v0 : col[r]);
            }
        }
        __syncthreads();
        if (tau != 0.0 && tid == 0 && c >= r0 && c < r1) col[c] = v0;  // reflector stored in place
        __syncthreads();
    }
    cl.sync();  // partial buffers are reused below
    if (J.Rt) {
        for (int e = tid; e < (r1 - r0) * s; e += kQrThreads) {
            int i = r0 + e % (r1 - r0), j = e / (r1 - r0);
            if (i >= s) continue;
            double v = 0.0;
            if (i < j) v = A[(int64_t)j * lda + i];
            else if (i == j) v = betas[i];
            J.Rt[(int64_t)i * s + j] = v;
            if (J.Rt2) {
                const float h = __double2float_rn(v);
                J.Rt2[(int64_t)i * s + j] = make_float2(h, __double2float_rn(v - (double)h));
            }
        }
    }
    if (!J.Q) return;
    double *Q = J.Q;
    const int64_t ldq = J.ldq;
    for (int e = tid; e < (r1 - r0) * s; e += kQrThreads) {
        int r = r0 + e % (r1 - r0), j = e / (r1 - r0);
        Q[(int64_t)j * ldq + r] = (r == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    int active = 0;
    for (int c = s - 1; c >= 0; --c) {
        const double tau = taus[c];
        if (tau == 0.0) continue;  // identical on every CTA of the cluster
        const double *v = A + (int64_t)c * lda;
        double *pb = dots + (active & 1) * s;
        ++active;
        const int rb = max(r0, c);
        for (int cc = c + warp; cc < s; cc += kNw) {
            const double *dst = Q + (int64_t)cc * ldq;
            double w = 0.0;
            for (int r = rb + lane; r < r1; r += 32) w += v[r] * dst[r];
            w = warp_sum(w);
            if (lane == 0) pb[cc] = w;
        }
        cl.sync();
        for (int cc = c + warp; cc < s; cc += kNw) {
            double w = 0.0;
            for (int k = 0; k < kCl; ++k) w += cl.map_shared_rank(pb, k)[cc];
            w *= tau;
            double *dst = Q + (int64_t)cc * ldq;
            for (int r = rb + lane; r < r1; r += 32) dst[r] -= w * v[r];
        }
        __syncthreads();
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD of M = R' (s x s): right rotations make the
// columns of M mutually orthogonal, M J = W S; S are the column norms and W
// the unit columns.  Output sorted by S descending (non-finite last).
struct SvdJob {
    const double *Rt;  // s x s input R' (ld s)
    double *work;      // s x s workspace (global-memory variant only)
    double *W;         // s x s output: unit left singular vectors of R', sorted
    double *S;         // s output singular values, descending
    int *rank;         // #{S > tau}, or -1 if any S is not finite
    int *sweeps;       // [0] FP64 sweeps, [1] FP32 sweeps, [2] FP64 pairs checked, [3] FP64 pairs rotated
    int s;
    double tau;        // absolute accuracy of the tile
    const float2 *Rt2; // R' as paired FP32 (the paired-FP32 precondition reads it), or null
};

// Fast approximate reciprocal and reciprocal square root of a double (the
// PTX approximation instructions); callers refine them where it matters.
__device__ __forceinline__ double rcp_approx(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}
__device__ __forceinline__ double rsqrt_approx(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// Squared norm of the first sdot entries of x (lanes stride 32; warp-uniform result).
// FP32 columns are read as pairs of entries per lane (8-byte shared-memory
// accesses, half the load instructions; the FP32 phase's columns hold 2 s
// entries and start on 8-byte boundaries).
template <class T>
__device__ __forceinline__ T col_norm2(const T *x, int sdot, int lane) {
    T a = 0;
    if constexpr (std::is_same<T, float>::value) {
        const float2 *x2 = reinterpret_cast<const float2 *>(x);
        for (int i = lane; 2 * i < sdot; i += 32) {
            const float2 v = x2[i];
            a = fmaf(v.x, v.x, a);
            if (2 * i + 1 < sdot) a = fmaf(v.y, v.y, a);
        }
    } else {
        for (int r = lane; r < sdot; r += 32) a = fma(x[r], x[r], a);
    }
    return warp_sum(a);
}

// Rotate columns x and y so that their first sdot entries become orthogonal;
// the rotation is applied to all srot entries (srot > sdot carries the
// accumulated rotations along).  nx, ny hold the squared norms of the two
// columns (first sdot entries) and are updated, so that a pair costs one dot
// product instead of three (the update is c^2 (a -+ 2 t g + t^2 b), exact for
// any t; a norm is recomputed when that formula cancels more than three
// digits).  Returns whether a rotation was applied.  Pairs with
// |x'y| <= tol |x| |y| (tol2 = tol^2) are left alone.
// FP64: the rotation angle only steers convergence, so t = tan(angle) comes
// from approximations; c = 1/sqrt(1 + t^2) is refined by two Newton steps for
// the reciprocal square root, y <- y (3 - x y^2) / 2, so that (c, c t) is
// orthogonal to working precision and the singular values are preserved.
template <class T>
__device__ __forceinline__ bool jacobi_rotate(T *x, T *y, T *nx, T *ny, int sdot, int srot, int lane, T tol2) {
    const T al = *nx, be = *ny;
    T ga = 0;
    if constexpr (std::is_same<T, float>::value) {
        const float2 *x2 = reinterpret_cast<const float2 *>(x), *y2 = reinterpret_cast<const float2 *>(y);
        for (int i = lane; 2 * i < sdot; i += 32) {
            const float2 u = x2[i], v = y2[i];
            ga = fmaf(u.x, v.x, ga);
            if (2 * i + 1 < sdot) ga = fmaf(u.y, v.y, ga);
        }
    } else {
        for (int r = lane; r < sdot; r += 32) ga = fma(x[r], y[r], ga);
    }
    ga = warp_sum(ga);
    if (ga == T(0) || ga * ga <= tol2 * (al * be)) return false;
    T c, sn, t;
    if constexpr (std::is_same<T, double>::value) {
        double rg = rcp_approx(2.0 * ga);
        rg = rg * fma(-2.0 * ga, rg, 2.0);
        const double zeta = (be - al) * rg, az = fabs(zeta);
        const double q = fma(zeta, zeta, 1.0);
        t = copysign(az < 1e150 ? rcp_approx(az + q * rsqrt_approx(q)) : 0.5 * rcp_approx(az), zeta);
        const double u = fma(t, t, 1.0);
        c = rsqrt_approx(u);
        c = c * fma(-0.5 * u * c, c, 1.5);
        c = c * fma(-0.5 * u * c, c, 1.5);
        sn = c * t;
    } else {
        // approximate reciprocals and square root: (c, c t) is orthogonal to
        // FP32 accuracy for any t, so only convergence depends on them
        const float zeta = __fdividef(be - al, 2.0f * ga), az = fabsf(zeta);
        if (az >= 1e18f) return false;  // t below FP32 resolution
        const float q = fmaf(zeta, zeta, 1.0f);
        t = copysignf(__fdividef(1.0f, az + q * rsqrtf(q)), zeta);
        c = rsqrtf(fmaf(t, t, 1.0f));
        sn = c * t;
    }
    if constexpr (std::is_same<T, float>::value) {
        float2 *x2 = reinterpret_cast<float2 *>(x), *y2 = reinterpret_cast<float2 *>(y);
        for (int i = lane; 2 * i < srot; i += 32) {  // srot is even in the FP32 phase
            const float2 a = x2[i], b = y2[i];
            x2[i] = make_float2(fmaf(c, a.x, -sn * b.x), fmaf(c, a.y, -sn * b.y));
            y2[i] = make_float2(fmaf(sn, a.x, c * b.x), fmaf(sn, a.y, c * b.y));
        }
    } else {
        for (int r = lane; r < srot; r += 32) {
            const T a = x[r], b = y[r];
            x[r] = fma(c, a, -sn * b);
            y[r] = fma(sn, a, c * b);
        }
    }
    const T c2 = c * c, tg = T(2) * t * ga, tt = t * t;
    T al2 = c2 * (al - tg + tt * be), be2 = c2 * (be + tg + tt * al);
    if (!(al2 > T(1e-3) * c2 * (al + tt * be))) al2 = col_norm2(x, sdot, lane);
    if (!(be2 > T(1e-3) * c2 * (be + tt * al))) be2 = col_norm2(y, sdot, lane);
    if (lane == 0) {
        *nx = al2;
        *ny = be2;
    }
    return true;
}

// Convergence threshold of a pair, squared: |x'y| <= 8 sqrt(s) u |x| |y|
// (u the unit roundoff of T), a few times the rounding error of the dot
// products, so that rounding alone never keeps a sweep alive.
template <class T>
__device__ __forceinline__ T jacobi_tol2(int s) {
    const T u = std::is_same<T, double>::value ? T(1.1102230246251565e-16) : T(5.9604644775390625e-8);
    const T tol = T(8) * sqrt((T)s) * u;
    return tol * tol;
}

// Sort key of a column norm: non-finite values sort last.
__device__ __forceinline__ double norm_key(double v) { return v <= 1.7e308 ? v : -1.0; }

// Round-robin tournament over 2C blocks: block held at position `pos` in
// global round g (position 0 stays, the others rotate), and its inverse.
__device__ __forceinline__ int block_at(int pos, int g, int nblk) {
    return pos == 0 ? 0 : 1 + (pos - 1 + g) % (nblk - 1);
}
__device__ __forceinline__ int pos_of(int blk, int g, int nblk) {
    return blk == 0 ? 0 : 1 + ((blk - 1 - g) % (nblk - 1) + (nblk - 1)) % (nblk - 1);
}

// Rotate all pairs between the two b-column blocks X (global block bx) and Y
// (by), and, if `inner`, the pairs within each of them.  Columns are srot
// apart within a block; NX, NY hold their squared norms.  Virtual columns
// (global index >= s) are zero and skipped.  Returns whether any rotation was
// applied by this thread's warp.
template <class T>
__device__ __forceinline__ bool jacobi_block_pairs(T *X, T *Y, T *NX, T *NY, int bx, int by, int b, int s, int srot,
                                                   bool inner, int lane, int warp, T tol2, int &nchk, int &nrot) {
    bool rot = false;
    if (inner) {
        const int bp = b + (b & 1);
        for (int ir = 0; ir < bp - 1; ++ir) {
            for (int pr = warp; pr < bp; pr += kNw) {  // bp/2 pairs per block, two blocks
                const int slot = pr / (bp / 2), q = pr % (bp / 2);
                const int a = (q == 0) ? 0 : 1 + (q - 1 + ir) % (bp - 1);
                const int c2 = 1 + (bp - 2 - q + ir) % (bp - 1);
                const int blk = slot ? by : bx;
                if (a >= b || c2 >= b || blk * b + max(a, c2) >= s) continue;
                T *base = slot ? Y : X;
                T *nrm = slot ? NY : NX;
                const int lo = min(a, c2), hi = max(a, c2);
                const bool r = jacobi_rotate(base + lo * srot, base + hi * srot, nrm + lo, nrm + hi, s, srot, lane, tol2);
                rot |= r;
                ++nchk;
                nrot += r;
            }
            __syncthreads();
        }
    }
    for (int k = 0; k < b; ++k) {
        for (int i = warp; i < b; i += kNw) {
            const int jy = (i + k) % b;
            const int gx = bx * b + i, gy = by * b + jy;
            if (gx >= s || gy >= s) continue;
            // the lower global index is the first column of the pair
            const bool r = gx < gy ? jacobi_rotate(X + i * srot, Y + jy * srot, NX + i, NY + jy, s, srot, lane, tol2)
                                   : jacobi_rotate(Y + jy * srot, X + i * srot, NY + jy, NX + i, s, srot, lane, tol2);
            rot |= r;
            ++nchk;
            nrot += r;
        }
        __syncthreads();
    }
    return rot;
}

// Squared norms of the 2b columns of a buffer (first s entries of each).
template <class T>
__device__ __forceinline__ void block_norms(const T *cols, T *nrm, int b, int s, int srot, int lane, int warp) {
    for (int q = warp; q < 2 * b; q += kNw) {
        const T v = col_norm2(cols + q * srot, s, lane);
        if (lane == 0) nrm[q] = v;
    }
    __syncthreads();
}

// Sweeps of the shared-memory block Jacobi: each CTA holds two blocks of b
// columns (srot elements each) and their squared norms in buffer cur
// (buf0 + cur * stride: slot 0, slot 1, then 2b norms); after each block
// round the CTAs pull their next blocks over DSMEM into the other buffer.
// Norms are recomputed at the start of every sweep.  Runs until a sweep
// rotates nothing or max_sweeps; g (global round) and cur are updated so
// that buffer cur holds the blocks of positions (rank, 2C - 1 - rank) at
// round g on return.  Returns the number of sweeps run.
template <int kCl, class T>
__device__ int jacobi_sweeps(cg::cluster_group &cl, T *buf0, int stride, int b, int s, int srot, int max_sweeps,
                             int &g, int &cur, int *s_flag, int *tally = nullptr) {
    int nchk = 0, nrot = 0;  // pairs checked and rotated by this warp (warp-uniform)
    constexpr int nblk = 2 * kCl;
    const int rank = (int)cl.block_rank(), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int px = rank, py = nblk - 1 - rank, bs = b * srot;
    const T tol2 = jacobi_tol2<T>(s);
    auto buf = [&](int k) { return buf0 + k * stride; };
    int nsweep = 0;
    bool done = false;
    for (int sweep = 0; sweep < max_sweeps && !done; ++sweep, ++nsweep) {
        if (tid == 0) s_flag[sweep & 1] = 0;
        block_norms(buf(cur), buf(cur) + 2 * bs, b, s, srot, lane, warp);
        for (int round = 0; round < nblk - 1; ++round, ++g) {
            const int bx = block_at(px, g, nblk), by = block_at(py, g, nblk);
            T *B = buf(cur);
            if (jacobi_block_pairs<T>(B, B + bs, B + 2 * bs, B + 2 * bs + b, bx, by, b, s, srot, round == 0, lane,
                                      warp, tol2, nchk, nrot) &&
                lane == 0)
                s_flag[sweep & 1] = 1;
            cl.sync();
            if (round == nblk - 2) {
                int any = 0;
#pragma unroll
                for (int k = 0; k < kCl; ++k) any |= cl.map_shared_rank(s_flag, k)[sweep & 1];
                if (!any) {
                    done = true;
                    break;
                }
            }
            // pull the blocks (and norms) of round g + 1 from their holders in
            // round g: kPull remote loads of each slot are issued before any
            // store (the compiler cannot tell the remote source from the
            // local destination, so a load-store loop waits out every round
            // trip)
            {
                const T *src[2];
                T *dst = buf(cur ^ 1);
                for (int slot = 0; slot < 2; ++slot) {
                    const int blk = block_at(slot ? py : px, g + 1, nblk);
                    const int p = pos_of(blk, g, nblk);
                    const int h = p < kCl ? p : nblk - 1 - p, hs = p < kCl ? 0 : 1;
                    src[slot] = cl.map_shared_rank(buf(cur), h) + hs * bs;
                    const T *ns = cl.map_shared_rank(buf(cur), h) + 2 * bs + hs * b;
                    for (int e = tid; e < b; e += kQrThreads) dst[2 * bs + slot * b + e] = ns[e];
                }
                constexpr int kPull = 4;
                for (int e0 = tid; e0 < bs; e0 += kPull * kQrThreads) {
                    T v[2][kPull];
#pragma unroll
                    for (int u = 0; u < kPull; ++u) {
                        const int e = e0 + u * kQrThreads;
                        v[0][u] = e < bs ? src[0][e] : T(0);
                        v[1][u] = e < bs ? src[1][e] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < kPull; ++u) {
                        const int e = e0 + u * kQrThreads;
                        if (e < bs) {
                            dst[e] = v[0][u];
                            dst[bs + e] = v[1][u];
                        }
                    }
                }
            }
            cur ^= 1;
            __syncthreads();
        }
    }
    if (tally && lane == 0) {
        atomicAdd(tally, nchk);
        atomicAdd(tally + 1, nrot);
    }
    return nsweep;
}

// Column norms, descending order over the whole matrix, and the output of the
// columns held in `cols` (global indices gx * b + j and gy * b + j).
// `all_nrm` must hold every column's norm on entry.
__device__ __forceinline__ void jacobi_emit(const SvdJob &J, const double *cols, int gx, int gy, int b,
                                            const double *all_nrm, int lane, int warp) {
    const int s = J.s;
    for (int q = warp; q < 2 * b; q += kNw) {
        const int slot = q / b, j = q % b, u = (slot ? gy : gx) * b + j;
        if (u >= s) continue;
        const double ku = norm_key(all_nrm[u]);
        int pos = 0;
        for (int w = lane; w < s; w += 32) {
            const double kw = norm_key(all_nrm[w]);
            pos += (kw > ku) || (kw == ku && w < u);
        }
        pos = __reduce_add_sync(0xFFFFFFFFu, pos);
        const double nv = all_nrm[u];
        const bool unit = nv > 0.0 && nv <= 1.7e308;
        const double *col = cols + q * s;
        const double inv = unit ? 1.0 / nv : 1.0;  // one division per column, not per entry
        for (int r = lane; r < s; r += 32) J.W[(int64_t)pos * s + r] = col[r] * inv;
        if (lane == 0) J.S[pos] = nv;
    }
}

__device__ void jacobi_rank(const SvdJob &J, const double *all_nrm, int sweeps, int sweeps32) {
    J.sweeps[0] = sweeps;
    J.sweeps[1] = sweeps32;
    J.sweeps[2] = J.sweeps[3] = 0;
    int r = 0;
    bool bad = false;
    for (int u = 0; u < J.s; ++u) {
        r += all_nrm[u] > J.tau;
        bad |= !(all_nrm[u] <= 1.7e308);
    }
    *J.rank = bad ? -1 : r;
}

constexpr int kMaxSweeps32 = 12;
constexpr int kRefineSteps = 3;  // FP64 Gram refinement steps after the FP32 sweeps

// Block Jacobi with the blocks in shared memory, in two precisions.
//  A. FP32 sweeps on fl32(M), M = R', carrying the accumulated rotations J
//     (each column holds s entries of M then s of J), until FP32 convergence.
//  B. M1 = M J in FP64 (M read from R', J from shared memory) into `work`.
//  C. FP64 sweeps on M1 until convergence; S, W from M1's columns.
// J is orthogonal to FP32 accuracy, so M1 = (M J_o)(I + E) with J_o
// orthogonal and |E| ~ 1e-7: a right multiplicative perturbation, under
// which every singular value of M1 is that of M times (1 + O(|E|)) and the
// dominant left singular subspace of M1 projects M with the error
// sigma_{r+1}(M) (1 + O(|E|)) (relative perturbation theory; Eisenstat and
// Ipsen 1995).  The FP32 sweeps do the bulk of the rotations on a pipe 64
// times faster than FP64; the FP64 phase then converges in a few sweeps.
// Shared memory: two buffers of two b x s blocks and 2b squared norms (FP64
// layout; the FP32 phase stores b x 2s floats per block in the same bytes),
// 2b local norms, s gathered norms.
// kMode: kJacFull runs A, B, C and writes W, S, rank; kJacPrecond runs A and
// B only (M1 left in `work` for the FP64 Gram refinement); kJacFinish runs C
// only, on the M1 found in `work`.
enum { kJacFull = 0, kJacPrecond = 1, kJacFinish = 2 };
template <int kCl, int kMode>
__global__ void __launch_bounds__(kQrThreads, 2) k_jacobi_sm(const SvdJob *__restrict__ jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ int s_flag[2];
    __shared__ int s_tally[2];  // FP64 phase: pairs checked, pairs rotated (this CTA)
    extern __shared__ double sm[];
    const SvdJob J = jobs[blockIdx.x / kCl];
    const int s = J.s, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nblk = 2 * kCl;
    const int b = (s + nblk - 1) / nblk, bs = b * s;
    const int stride = 2 * bs + 2 * b;  // one buffer: two blocks, 2b norms (FP64 layout)
    if (tid == 0) s_tally[0] = s_tally[1] = 0;
    double *nrm_loc = sm + 2 * stride, *all_nrm = nrm_loc + 2 * b;
    const int px = rank, py = nblk - 1 - rank;
    int g = 0, cur = 0, sw32 = 0;
    if (kMode != kJacFinish) {
    // A. FP32 phase (the same buffers hold b x 2s floats per block)
    float *f0 = reinterpret_cast<float *>(sm);
    const int s2 = 2 * s, bsf = b * s2, stride_f = 2 * bsf + 2 * b;
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = block_at(slot ? py : px, 0, nblk);
        float *dst = f0 + slot * bsf;
        for (int e = tid; e < bsf; e += kQrThreads) {
            const int u = blk * b + e / s2, r = e % s2;
            float v = 0.0f;
            if (u < s) {
                if (r >= s) v = r - s == u ? 1.0f : 0.0f;
                else v = J.Rt2 ? J.Rt2[(int64_t)u * s + r].x : (float)J.Rt[(int64_t)u * s + r];
            }
            dst[e] = v;
        }
    }
    __syncthreads();
    sw32 = jacobi_sweeps<kCl, float>(cl, f0, stride_f, b, s, s2, kMaxSweeps32, g, cur, s_flag);
    // B. M1 = M J for the held columns, 8 at a time; rows i = tid, tid + 256.
    // With the paired copy of M (paired-FP32 paths) the products run in
    // float-float arithmetic on the FP32 pipe (J is exact in FP32; M1 then
    // carries ~1e-14 of |M|, below the thresholds of those paths); else in
    // FP64.  Warps whose rows all lie past s, and the second row when
    // s <= 256, issue nothing (an FP64 warp instruction costs the same with
    // no lane active).
    {
        const float *F = f0 + cur * stride_f;
        const int gx = block_at(px, g, nblk), gy = block_at(py, g, nblk);
        const bool rows2 = s > kQrThreads, live = warp * 32 < s;
        for (int q0 = 0; q0 < 2 * b && live; q0 += 8) {
            double out[8][2];
            if (J.Rt2) {
                float h[8][2], l[8][2];
#pragma unroll
                for (int a = 0; a < 8; ++a) h[a][0] = h[a][1] = l[a][0] = l[a][1] = 0.0f;
                for (int k = 0; k < s; ++k) {
                    const float2 m0 = tid < s ? J.Rt2[(int64_t)k * s + tid] : make_float2(0.f, 0.f);
                    const float2 m1 = rows2 && tid + kQrThreads < s ? J.Rt2[(int64_t)k * s + tid + kQrThreads]
                                                                    : make_float2(0.f, 0.f);
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const int q = q0 + a;
                        const float jk = q < 2 * b ? F[q * s2 + s + k] : 0.0f;
                        df_fma(m0.x, m0.y, jk, 0.0f, h[a][0], l[a][0]);
                        if (rows2) df_fma(m1.x, m1.y, jk, 0.0f, h[a][1], l[a][1]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    out[a][0] = (double)h[a][0] + (double)l[a][0];
                    out[a][1] = (double)h[a][1] + (double)l[a][1];
                }
            } else {
#pragma unroll
                for (int a = 0; a < 8; ++a) out[a][0] = out[a][1] = 0.0;
                for (int k = 0; k < s; ++k) {
                    const double m0 = tid < s ? J.Rt[(int64_t)k * s + tid] : 0.0;
                    const double m1 = rows2 && tid + kQrThreads < s ? J.Rt[(int64_t)k * s + tid + kQrThreads] : 0.0;
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const int q = q0 + a;
                        const double jk = q < 2 * b ? (double)F[q * s2 + s + k] : 0.0;
                        out[a][0] = fma(m0, jk, out[a][0]);
                        if (rows2) out[a][1] = fma(m1, jk, out[a][1]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int q = q0 + a;
                if (q >= 2 * b) break;
                const int u = (q < b ? gx : gy) * b + q % b;
                if (u >= s) continue;
                if (tid < s) J.work[(int64_t)u * s + tid] = out[a][0];
                if (tid + kQrThreads < s) J.work[(int64_t)u * s + tid + kQrThreads] = out[a][1];
            }
        }
    }
    cl.sync();  // M1 complete; no CTA reads another's FP32 blocks any more
    if (kMode == kJacPrecond) {
        if (rank == 0 && tid == 0) {
            J.sweeps[0] = 0;
            J.sweeps[1] = sw32;
            J.sweeps[2] = J.sweeps[3] = 0;
        }
        return;
    }
    }  // kMode != kJacFinish
    // C. FP64 phase on M1, starting from the same block positions
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = block_at(slot ? py : px, g, nblk);
        double *dst = sm + slot * bs;
        for (int e = tid; e < bs; e += kQrThreads) {
            const int u = blk * b + e / s;
            dst[e] = u < s ? J.work[(int64_t)u * s + e % s] : 0.0;
        }
    }
    __syncthreads();
    cur = 0;
    const int sw64 = jacobi_sweeps<kCl, double>(cl, sm, stride, b, s, s, kMaxSweeps, g, cur, s_flag, s_tally);
    double *D = sm + cur * stride;
    const int gx = block_at(px, g, nblk), gy = block_at(py, g, nblk);
    for (int q = warp; q < 2 * b; q += kNw) {
        const double *col = D + q * s;
        double v = 0.0;
        for (int r = lane; r < s; r += 32) v = fma(col[r], col[r], v);
        v = warp_sum(v);
        if (lane == 0) nrm_loc[q] = sqrt(v);
    }
    cl.sync();
    for (int e = tid; e < 2 * b * kCl; e += kQrThreads) {
        const int h = e / (2 * b), q = e % (2 * b), slot = q / b, j = q % b;
        const int u = block_at(slot ? nblk - 1 - h : h, g, nblk) * b + j;
        if (u < s) all_nrm[u] = cl.map_shared_rank(nrm_loc, h)[q];
    }
    __syncthreads();
    jacobi_emit(J, D, gx, gy, b, all_nrm, lane, warp);
    if (rank == 0 && tid == 0) {
        jacobi_rank(J, all_nrm, sw64, sw32);
        int chk = 0, rot = 0;
        for (int k = 0; k < kCl; ++k) {
            chk += cl.map_shared_rank(s_tally, k)[0];
            rot += cl.map_shared_rank(s_tally, k)[1];
        }
        J.sweeps[2] = chk;
        J.sweeps[3] = rot;
    }
    cl.sync();  // no CTA leaves while another may still read its norms or tallies
}

// FP64 Gram refinement of M1 (the columns of which are orthogonal to FP32
// accuracy after the preconditioning sweeps).  With G = M1'M1, every pair
// (i < j) gets its one-sided Jacobi angle t_ij from (G_ii, G_jj, G_ij), and
// all pairs are applied at once: M1 <- M1 (I + A), A_ij = t_ij, A_ji = -t_ij.
// For simple singular values this is a Newton-type step that squares the
// pairwise cosines |G_ij| / sqrt(G_ii G_jj) (~1e-6 -> ~1e-10 -> below the
// FP64 threshold in three steps); I + A is orthogonal to second order, a
// right multiplicative perturbation that moves the singular values by O(|A|^2)
// relative.  Pairs of two columns below 0.1 tau are skipped: their mutual
// orthogonality decides neither the rank nor the kept singular vectors.
// off[0] receives the largest cosine over the other pairs (as ordered bits).
struct RefineJob {
    const double *G;   // s x s Gram matrix (ld s)
    double *IA;        // s x s output I + A (ld s)
    unsigned long long *off;
    double tail2;      // (0.1 tau)^2
    int s;
};

__global__ void k_refine_angles(const RefineJob *__restrict__ jobs) {
    const RefineJob J = jobs[blockIdx.y];
    const int s = J.s;
    double worst = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s * s; e += gridDim.x * blockDim.x) {
        const int i = e % s, j = e / s;
        double v = (i == j) ? 1.0 : 0.0;
        if (i != j) {
            const int a = min(i, j), b = max(i, j);
            const double al = J.G[(int64_t)a * s + a], be = J.G[(int64_t)b * s + b], ga = J.G[(int64_t)b * s + a];
            if (!(al < J.tail2 && be < J.tail2) && ga != 0.0) {
                const double zeta = (be - al) / (2.0 * ga);
                const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                v = (i == a) ? t : -t;
                const double c = fabs(ga) / sqrt(al * be);
                worst = c == c ? fmax(worst, c) : INFINITY;
            }
        }
        J.IA[e] = v;
    }
    for (int o = 16; o; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xFFFFFFFFu, worst, o));
    if ((threadIdx.x & 31) == 0 && worst > 0.0) atomicMax(J.off, (unsigned long long)__double_as_longlong(worst));
}

// Singular values and vectors of the refined M1 (one CTA per job): column
// norms, descending order (non-finite last), W = unit columns, S, and the
// rank #{S > tau}: -1 for non-finite values, -2 when the refinement had not
// converged (the caller then finishes with FP64 Jacobi sweeps).
struct EmitJob {
    const double *X;   // s x s refined M1 (ld s)
    double *W;
    double *S;
    int *rank;
    const unsigned long long *off;
    int s;
    double tau;
};

__global__ void __launch_bounds__(kQrThreads) k_svd_emit(const EmitJob *__restrict__ jobs) {
    extern __shared__ double nrm[];
    const EmitJob J = jobs[blockIdx.x];
    const int s = J.s, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int u = warp; u < s; u += kNw) {
        const double v = col_norm2(J.X + (int64_t)u * s, s, lane);
        if (lane == 0) nrm[u] = sqrt(v);
    }
    __syncthreads();
    for (int u = warp; u < s; u += kNw) {
        const double ku = norm_key(nrm[u]);
        int pos = 0;
        for (int w = lane; w < s; w += 32) {
            const double kw = norm_key(nrm[w]);
            pos += (kw > ku) || (kw == ku && w < u);
        }
        pos = __reduce_add_sync(0xFFFFFFFFu, pos);
        const double nv = nrm[u];
        const bool unit = nv > 0.0 && nv <= 1.7e308;
        const double *col = J.X + (int64_t)u * s;
        const double inv = unit ? 1.0 / nv : 1.0;  // one division per column, not per entry
        for (int r = lane; r < s; r += 32) J.W[(int64_t)pos * s + r] = col[r] * inv;
        if (lane == 0) J.S[pos] = nv;
    }
    if (tid == 0) {
        int r = 0;
        bool bad = false;
        for (int u = 0; u < s; ++u) {
            r += nrm[u] > J.tau;
            bad |= !(nrm[u] <= 1.7e308);
        }
        const double off = __longlong_as_double((long long)*J.off);
        const double tol = 8.0 * sqrt((double)s) * 1.1102230246251565e-16;
        *J.rank = bad ? -1 : (off > tol ? -2 : r);
    }
}

static size_t jacobi_sm_bytes(int s, int csize) {
    const int b = (s + 2 * csize - 1) / (2 * csize);
    return ((size_t)4 * b * s + 6 * b + s) * sizeof(double);
}

// Block Jacobi with the matrix in global memory (L2): the two blocks of a
// round are staged in shared memory and written back before the cluster
// barrier.  Shared memory: two b x s blocks, their 2b squared norms, s norms.
template <int kCl>
__global__ void __launch_bounds__(kQrThreads) k_jacobi_gm(const SvdJob *__restrict__ jobs) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ int s_flag[2];
    extern __shared__ double sm[];
    const SvdJob J = jobs[blockIdx.x / kCl];
    const int s = J.s, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nblk = 2 * kCl;
    const int b = (s + nblk - 1) / nblk, bs = b * s;
    double *Ab = sm, *Nb = sm + 2 * bs, *all_nrm = Nb + 2 * b;
    double *A = J.work;
    for (int e = rank * kQrThreads + tid; e < s * s; e += kCl * kQrThreads) __stcg(A + e, J.Rt[e]);
    cl.sync();
    const int px = rank, py = nblk - 1 - rank;
    int g = 0, nsweep = 0;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        ++nsweep;
        if (tid == 0) s_flag[sweep & 1] = 0;
        __syncthreads();
        for (int round = 0; round < nblk - 1; ++round, ++g) {
            const int bx = block_at(px, g, nblk), by = block_at(py, g, nblk);
            for (int e = tid; e < 2 * bs; e += kQrThreads) {
                const int slot = e / bs, u = (slot ? by : bx) * b + (e % bs) / s;
                Ab[e] = u < s ? __ldcg(A + (int64_t)u * s + e % s) : 0.0;
            }
            __syncthreads();
            block_norms(Ab, Nb, b, s, s, lane, warp);
            int nchk = 0, nrot = 0;
            if (jacobi_block_pairs<double>(Ab, Ab + bs, Nb, Nb + b, bx, by, b, s, s, round == 0, lane, warp,
                                           jacobi_tol2<double>(s), nchk, nrot) &&
                lane == 0)
                s_flag[sweep & 1] = 1;
            for (int e = tid; e < 2 * bs; e += kQrThreads) {
                const int slot = e / bs, u = (slot ? by : bx) * b + (e % bs) / s;
                if (u < s) __stcg(A + (int64_t)u * s + e % s, Ab[e]);
            }
            cl.sync();
        }
        int any = 0;
        for (int k = 0; k < kCl; ++k) any |= cl.map_shared_rank(s_flag, k)[sweep & 1];
        if (!any) break;
    }
    // every CTA computes all norms; each writes its positions' columns
    for (int u = warp; u < s; u += kNw) {
        double v = 0.0;
        for (int r = lane; r < s; r += 32) {
            const double x = __ldcg(A + (int64_t)u * s + r);
            v = fma(x, x, v);
        }
        v = warp_sum(v);
        if (lane == 0) all_nrm[u] = sqrt(v);
    }
    __syncthreads();
    const int gx = block_at(px, g, nblk), gy = block_at(py, g, nblk);
    for (int e = tid; e < 2 * bs; e += kQrThreads) {
        const int slot = e / bs, u = (slot ? gy : gx) * b + (e % bs) / s;
        Ab[e] = u < s ? __ldcg(A + (int64_t)u * s + e % s) : 0.0;
    }
    __syncthreads();
    jacobi_emit(J, Ab, gx, gy, b, all_nrm, lane, warp);
    if (rank == 0 && tid == 0) jacobi_rank(J, all_nrm, nsweep, 0);
    cl.sync();  // no CTA leaves while another may still read its flag
}

static size_t jacobi_gm_bytes(int s, int csize) {
    const int b = (s + 2 * csize - 1) / (2 * csize);
    return ((size_t)2 * b * s + 2 * b + s) * sizeof(double);
}

// ---------------------------------------------------------------------------
// Launch helpers.

template <class K, class... Args>
static void launch_cluster(K kernel, int csize, int nclusters, int threads, size_t smem, cudaStream_t st,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * csize));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
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

// Dynamic shared memory a kernel may use: the device's opt-in per-block limit
// minus the kernel's static shared memory (the attribute is raised once).
static size_t smem_cap(const void *kernel) {
    static std::mutex mu;
    static std::map<const void *, size_t> caps;
    std::lock_guard<std::mutex> lock(mu);
    auto it = caps.find(kernel);
    if (it != caps.end()) return it->second;
    int dev = 0, optin = 0;
    TLR_CUDA_TRY(cudaGetDevice(&dev));
    TLR_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    TLR_CUDA_TRY(cudaFuncGetAttributes(&fa, kernel));
    size_t cap = (size_t)optin - fa.sharedSizeBytes;
    TLR_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
    caps[kernel] = cap;
    return cap;
}

// Whether clusters of 16 CTAs (a non-portable size) can run on this device.
static bool cluster16_ok() {
    static std::once_flag once;
    static int state = 0;
    std::call_once(once, [] {
        const void *k16[] = {(const void *)k_qr_sm<16, false>, (const void *)k_qr_sm<16, true>, (const void *)k_qr_gm<16>, (const void *)k_jacobi_sm<16, kJacFull>,
                             (const void *)k_jacobi_sm<16, kJacPrecond>, (const void *)k_jacobi_sm<16, kJacFinish>,
                             (const void *)k_jacobi_gm<16>};
        bool ok = true;
        for (const void *k : k16)
            ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
        if (ok) {
            // one cluster of 16 CTAs that each fill an SM's shared memory must fit
            const size_t need = std::min(smem_cap((const void *)k_qr_sm<16, false>), smem_cap((const void *)k_jacobi_sm<16, kJacFull>));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(kQrThreads);
            cfg.dynamicSmemBytes = need;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 16;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n1 = 0, n2 = 0;
            cudaLaunchConfig_t cfq = cfg;
            cfq.blockDim = dim3(kQrSmThreads);
            if (cudaOccupancyMaxActiveClusters(&n1, k_qr_sm<16, false>, &cfq) == cudaSuccess &&
                cudaOccupancyMaxActiveClusters(&n2, k_jacobi_sm<16, kJacFull>, &cfg) == cudaSuccess && n1 > 0 && n2 > 0)
                state = 1;
        }
        cudaGetLastError();  // clear any error of the queries
    });
    return state == 1;
}

// Cluster sizes by sample size (the context's rank buckets): the panel work
// per column shrinks with the cluster, the barrier count does not, so small
// samples use small clusters.
static int bucket_size(const int32_t *edge, const int32_t *size, int s) {
    for (int b = 0; b + 1 < kBuckets; ++b)
        if (s <= edge[b]) return size[b];
    return size[kBuckets - 1];
}
static int qr_cluster(const tlr_ctx *ctx, int s) { return bucket_size(ctx->buckets.qr_edge, ctx->buckets.qr_size, s); }
static int svd_cluster(const tlr_ctx *ctx, int s) {
    return bucket_size(ctx->buckets.svd_edge, ctx->buckets.svd_size, s);
}

using QrKernel = void (*)(const QrJob *);
using SvdKernel = void (*)(const SvdJob *);

template <bool kDf>
static QrKernel qr_sm_kernel_t(int c) {
    switch (c) {
    case 1: return k_qr_sm<1, kDf>;
    case 2: return k_qr_sm<2, kDf>;
    case 4: return k_qr_sm<4, kDf>;
    case 8: return k_qr_sm<8, kDf>;
    default: return k_qr_sm<16, kDf>;
    }
}
static QrKernel qr_sm_kernel(int c, bool df) { return df ? qr_sm_kernel_t<true>(c) : qr_sm_kernel_t<false>(c); }
template <int kMode>
static SvdKernel svd_sm_kernel_m(int c) {
    switch (c) {
    case 1: return k_jacobi_sm<1, kMode>;
    case 2: return k_jacobi_sm<2, kMode>;
    case 4: return k_jacobi_sm<4, kMode>;
    case 8: return k_jacobi_sm<8, kMode>;
    default: return k_jacobi_sm<16, kMode>;
    }
}
static SvdKernel svd_sm_kernel(int c, int mode) {
    return mode == kJacPrecond ? svd_sm_kernel_m<kJacPrecond>(c)
                               : (mode == kJacFinish ? svd_sm_kernel_m<kJacFinish>(c) : svd_sm_kernel_m<kJacFull>(c));
}

// One launch per (kernel, cluster size) class, with the class's largest
// shared-memory need.  The classes run concurrently, each on its own
// high-priority stream (forked from and joined back to the calling stream),
// largest clusters first: a column's compression then costs its slowest
// class, not the sum.
template <class Job, class K>
struct LaunchClass {
    K kernel;
    int csize;
    size_t smem = 0;
    std::vector<Job> jobs;
    int threads = kQrThreads;
};

// Events around the launch of one class (profiling).
struct ClassTiming {
    int csize = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static cudaEvent_t pooled_event(tlr_ctx *ctx, size_t &used) {
    while (ctx->cls_time_events.size() <= used) {
        cudaEvent_t e;
        TLR_CUDA_TRY(cudaEventCreate(&e));
        ctx->cls_time_events.push_back(e);
    }
    return ctx->cls_time_events[used++];
}

template <class Job, class K, class... Extra>
static void launch_classes(tlr_ctx *ctx, cudaStream_t st, std::vector<LaunchClass<Job, K>> &cls,
                           ClassTiming *timing, Extra... extra) {
    std::vector<LaunchClass<Job, K> *> use;
    for (auto &c : cls)
        if (!c.jobs.empty()) use.push_back(&c);
    std::stable_sort(use.begin(), use.end(), [](const LaunchClass<Job, K> *a, const LaunchClass<Job, K> *b) {
        return a->csize > b->csize;
    });
    // descriptors go up on the calling stream, before the fork
    std::vector<const Job *> dj;
    for (auto *c : use) dj.push_back((const Job *)stage_push(ctx, c->jobs.data(), c->jobs.size() * sizeof(Job), st));
    if (use.empty()) return;
    if ((int)use.size() > tlr_ctx::kClassEvents) throw make_error(TLR_ERR_ARG, "too many launch classes");
    TLR_CUDA_TRY(cudaEventRecord(ctx->cls_fork, st));
    for (size_t k = 0; k < use.size(); ++k) {
        cudaStream_t cs = ctx->cls_stream[k % tlr_ctx::kClassStreams];
        TLR_CUDA_TRY(cudaStreamWaitEvent(cs, ctx->cls_fork, 0));
        const bool timed = timing && timing->csize == use[k]->csize;
        if (timed) TLR_CUDA_TRY(cudaEventRecord(timing->e0, cs));
        launch_cluster(use[k]->kernel, use[k]->csize, (int)use[k]->jobs.size(), use[k]->threads, use[k]->smem, cs, dj[k],
                       extra...);
        if (timed) TLR_CUDA_TRY(cudaEventRecord(timing->e1, cs));
        TLR_CUDA_TRY(cudaEventRecord(ctx->cls_join[k], cs));
    }
    if (timing) {  // a class that did not run leaves the events unrecorded
        bool ran = false;
        for (auto *c : use) ran |= (c->csize == timing->csize);
        if (!ran) timing->csize = 0;
    }
    for (size_t k = 0; k < use.size(); ++k) TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->cls_join[k], 0));
}

template <class Job, class K>
static void add_to_class(std::vector<LaunchClass<Job, K>> &cls, K kernel, int csize, size_t smem, const Job &j,
                         int threads = kQrThreads) {
    for (auto &c : cls)
        if (c.kernel == kernel && c.csize == csize) {
            c.smem = std::max(c.smem, smem);
            c.jobs.push_back(j);
            return;
        }
    LaunchClass<Job, K> c{kernel, csize, smem, {j}, threads};
    cls.push_back(c);
}

// QR stage for a list of jobs.  `copy[u]` (k x s, may alias nothing) is
// scratch for jobs that fall back to the in-place global-memory kernel when
// the input must survive (R-only factorisations).
static void qr_launch(tlr_ctx *ctx, cudaStream_t st, const std::vector<QrJob> &jobs, const std::vector<double *> &copy,
                      bool df) {
    const bool big = cluster16_ok();
    std::vector<LaunchClass<QrJob, QrKernel>> cls;
    for (size_t u = 0; u < jobs.size(); ++u) {
        QrJob J = jobs[u];
        int c = qr_cluster(ctx, J.s);
        if (c == 16 && !big) c = 8;
        int top = big ? 16 : 8;
        while (c < top && qr_sm_bytes(J.m, J.s, c) > smem_cap((const void *)qr_sm_kernel(c, df))) c *= 2;
        QrKernel k = qr_sm_kernel(c, df);
        size_t bytes = qr_sm_bytes(J.m, J.s, c);
        if (bytes <= smem_cap((const void *)k)) {
            add_to_class(cls, k, c, bytes, J, kQrSmThreads);
            continue;
        }
        // global-memory fallback: factorises its input in place
        if (!J.Q) {
            TLR_CUDA_TRY(cudaMemcpy2DAsync(copy[u], (size_t)J.m * sizeof(double), J.A, (size_t)J.lda * sizeof(double),
                                           (size_t)J.m * sizeof(double), J.s, cudaMemcpyDeviceToDevice, st));
            J.A = copy[u];
            J.lda = J.m;
        }
        add_to_class(cls, big ? (QrKernel)k_qr_gm<16> : (QrKernel)k_qr_gm<8>, top, 6 * (size_t)J.s * sizeof(double),
                     J);
        ctx->comp_stats[5] += 1;
    }
    launch_classes(ctx, st, cls, (ClassTiming *)nullptr);
}

// The SVD stage.  csize_of[u] receives the cluster size job u ran on (0 for
// the global-memory variant); `timing` (optional) times one cluster size.
static void svd_launch(tlr_ctx *ctx, cudaStream_t st, const std::vector<SvdJob> &jobs, std::vector<int> &csize_of,
                       ClassTiming *timing, int mode) {
    csize_of.assign(jobs.size(), 0);
    const bool big = cluster16_ok();
    const int top = big ? 16 : 8;
    std::vector<LaunchClass<SvdJob, SvdKernel>> cls;
    for (size_t u = 0; u < jobs.size(); ++u) {
        const SvdJob &J = jobs[u];
        int c = svd_cluster(ctx, J.s);
        if (c > top) c = top;
        while (c < top && jacobi_sm_bytes(J.s, c) > smem_cap((const void *)svd_sm_kernel(c, mode))) c = std::max(2 * c, 4);
        SvdKernel k = svd_sm_kernel(c, mode);
        size_t bytes = jacobi_sm_bytes(J.s, c);
        if (bytes <= smem_cap((const void *)k)) {
            add_to_class(cls, k, c, bytes, J);
            csize_of[u] = c;
            continue;
        }
        SvdKernel kg = big ? (SvdKernel)k_jacobi_gm<16> : (SvdKernel)k_jacobi_gm<8>;
        bytes = jacobi_gm_bytes(J.s, top);
        if (bytes > smem_cap((const void *)kg)) throw make_error(TLR_ERR_ARG, "sample size %d too large for this device", J.s);
        add_to_class(cls, kg, top, bytes, J);
        ctx->comp_stats[6] += 1;
    }
    launch_classes(ctx, st, cls, timing);
}

__global__ void k_gaussian(double *__restrict__ a, int64_t count, uint64_t seed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    auto mix = [](uint64_t z) {
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    uint64_t u1 = mix(seed ^ (2 * (uint64_t)i)), u2 = mix(seed ^ (2 * (uint64_t)i + 1));
    double a1 = ((double)(u1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double a2 = (double)(u2 >> 11) * (1.0 / 9007199254740992.0);
    a[i] = sqrt(-2.0 * log(a1)) * cospi(2.0 * a2);
}

void ensure_omega(tlr_ctx *ctx, cudaStream_t s) {
    if (ctx->d_omega) return;
    ctx->omega_rows = kMaxTile;
    ctx->omega_cols = kMaxSample;
    int64_t cnt = (int64_t)ctx->omega_rows * ctx->omega_cols;
    TLR_CUDA_TRY(cudaMalloc(&ctx->d_omega, cnt * sizeof(double)));
    TLR_CUDA_TRY(cudaMalloc(&ctx->d_omega2, cnt * sizeof(float2)));
    launch(k_gaussian, (unsigned)ceil_div(cnt, 256), 256, 0, s, ctx->d_omega, cnt, 0x243F6A8885A308D3ull);
    TLR_CHECK_LAUNCH();
    split_f2(s, ctx->d_omega, ctx->omega_rows, ctx->omega_rows, ctx->omega_cols, ctx->d_omega2);
}

void compress_jobs(tlr_ctx *ctx, cudaStream_t st, std::vector<CompressJob> &jobs, std::vector<int> &ranks,
                   std::vector<int> &fail_order, bool df, const std::function<void()> &overlap, const GrowSlot &grow,
                   bool tc) {
    const bool dfp = df && !tc;  // paired-FP32 operand copies for the products
    bool overlapped = false;
    ensure_omega(ctx, st);
    // profiling marks between the sub-steps of each adaptive round, from a
    // pool that is not reused before compress_profile_collect reads it
    std::vector<cudaEvent_t> ev;
    auto cmark = [&]() {
        if (!ctx->profile) return;
        const size_t k = ctx->comp_used++;
        while (ctx->comp_events.size() <= k) {
            cudaEvent_t e;
            TLR_CUDA_TRY(cudaEventCreate(&e));
            ctx->comp_events.push_back(e);
        }
        TLR_CUDA_TRY(cudaEventRecord(ctx->comp_events[k], st));
        ev.push_back(ctx->comp_events[k]);
    };
    // 8 marks per round: start, after sampling, QR of Y, projection, QR of B,
    // SVD, host decision, U/V; the complete rounds are handed on to
    // compress_profile_collect (waiting for them here would hold the host
    // until this call's last products end, and the stream that takes the
    // next launches would idle)
    struct Flush {
        tlr_ctx *ctx;
        std::vector<cudaEvent_t> &ev;
        ~Flush() {
            if (!ctx->profile) return;
            ctx->comp_pending.insert(ctx->comp_pending.end(), ev.begin(), ev.begin() + (ev.size() / 8) * 8);
        }
    } flush{ctx, ev};
    const int nj = (int)jobs.size();
    ranks.assign(nj, 0);
    fail_order.clear();
    std::vector<int> sz(nj), pending;
    for (int q = 0; q < nj; ++q) {
        const CompressJob &J = jobs[q];
        int full = std::min(J.m, J.k);
        int g = std::max(32, ((J.s_guess + kOversample + 7) / 8) * 8);
        sz[q] = std::min(full, std::min(g, kMaxSample));
        if (full > 0) pending.push_back(q);
    }
    const double *omega = ctx->d_omega;
    const int ldo = ctx->omega_rows;
    while (!pending.empty()) {
        const size_t np = pending.size();
        // workspace offsets (doubles)
        std::vector<int64_t> oY(np), oQ(np), oB(np), oC(np), oR(np), oW(np), oK(np), oS(np), oQ2(np), oX2(np), oG(np),
            oIA(np), oR2(np), oB2(np), oW2(np);
        std::vector<int> ps(np);
        int64_t tot = 0;
        auto take = [&](int64_t cnt) { int64_t o = tot; tot += (cnt + 31) & ~31LL; return o; };
        for (size_t u = 0; u < np; ++u) {
            const CompressJob &J = jobs[pending[u]];
            int s = sz[pending[u]];
            ps[u] = s;
            oY[u] = take((int64_t)J.m * s);
            oQ[u] = take((int64_t)J.m * s);
            oB[u] = take((int64_t)J.k * s);
            oC[u] = take((int64_t)J.k * s);
            oR[u] = take((int64_t)s * s);
            oW[u] = take((int64_t)s * s);
            oK[u] = take((int64_t)s * s);
            oS[u] = take(s);
            oQ2[u] = dfp ? take((int64_t)J.m * s) : 0;  // float2, one double each
            oX2[u] = take((int64_t)s * s);
            oG[u] = take((int64_t)s * s);
            oIA[u] = take((int64_t)s * s);
            oR2[u] = df ? take((int64_t)s * s) : 0;  // float2, one double each
            oB2[u] = dfp ? take((int64_t)J.k * s) : 0;
            oW2[u] = dfp ? take((int64_t)s * s) : 0;
        }
        DevBuf ws(tot * sizeof(double) + np * sizeof(unsigned long long) + 5 * np * sizeof(int) + 256, st);
        double *W = ws.as<double>();
        unsigned long long *d_off = (unsigned long long *)(W + tot);
        int *d_rank = (int *)(d_off + np);
        cmark();
        // 1. Y = T Omega_s
        std::vector<GemmProb> g1;
        for (size_t u = 0; u < np; ++u) {
            const CompressJob &J = jobs[pending[u]];
            GemmProb a{};
            a.A = J.T; a.lda = J.ldt; a.m = J.m; a.k = J.k;
            a.B = omega; a.ldb = ldo; a.n = ps[u];
            a.C = W + oY[u]; a.ldc = J.m;
            a.A2 = J.T2; a.B2 = ctx->d_omega2;
            g1.push_back(a);
        }
        if (tc) gemm_tc(ctx, st, false, false, g1, 1.0, 0.0);
        else gemm_batched(ctx, st, false, false, g1, 1.0, 0.0, df);
        cmark();
        // 2. Q = orth(Y)
        std::vector<QrJob> q1(np);
        std::vector<double *> scratch(np);
        for (size_t u = 0; u < np; ++u) {
            const CompressJob &J = jobs[pending[u]];
            q1[u] = QrJob{W + oY[u], J.m, W + oQ[u], J.m, nullptr, J.m, ps[u]};
            scratch[u] = W + oC[u];
        }
        qr_launch(ctx, st, q1, scratch, df);
        if (dfp) {
            std::vector<SplitDesc> sd(np);
            for (size_t u = 0; u < np; ++u)
                sd[u] = SplitDesc{W + oQ[u], (float2 *)(W + oQ2[u]), jobs[pending[u]].m, jobs[pending[u]].m, ps[u]};
            split_f2_batched(ctx, st, sd);
        }
        cmark();
        // 3. B = T' Q (kept), R' of B = Q2 R
        std::vector<GemmProb> g2;
        for (size_t u = 0; u < np; ++u) {
            const CompressJob &J = jobs[pending[u]];
            GemmProb a{};
            a.A = J.T; a.lda = J.ldt; a.m = J.k; a.k = J.m;
            a.B = W + oQ[u]; a.ldb = J.m; a.n = ps[u];
            a.C = W + oB[u]; a.ldc = J.k;
            a.A2 = J.T2; a.B2 = (const float2 *)(W + oQ2[u]);
            g2.push_back(a);
        }
        if (tc) gemm_tc(ctx, st, true, false, g2, 1.0, 0.0);
        else gemm_batched(ctx, st, true, false, g2, 1.0, 0.0, df);
        cmark();
        std::vector<QrJob> q2(np);
        for (size_t u = 0; u < np; ++u) {
            const CompressJob &J = jobs[pending[u]];
            q2[u] = QrJob{W + oB[u], J.k, nullptr, 0, W + oR[u], J.k, ps[u], df ? (float2 *)(W + oR2[u]) : nullptr};
        }
        qr_launch(ctx, st, q2, scratch, df);
        cmark();
        // 4. SVD of R'
        std::vector<SvdJob> sv(np);
        for (size_t u = 0; u < np; ++u)
            sv[u] = SvdJob{W + oR[u], W + oK[u], W + oW[u], W + oS[u], d_rank + u, d_rank + np + 4 * u, ps[u],
                           jobs[pending[u]].tau, df ? (const float2 *)(W + oR2[u]) : nullptr};
        std::vector<int> svd_csize;
        ClassTiming t16;
        size_t ev_used = 0;
        if (ctx->profile) {
            t16.csize = 16;
            t16.e0 = pooled_event(ctx, ev_used);
            t16.e1 = pooled_event(ctx, ev_used);
        }
        svd_launch(ctx, st, sv, svd_csize, ctx->profile ? &t16 : nullptr, kJacPrecond);
        // FP64 Gram refinement (batched over the tiles), then W, S and the rank
        std::vector<double *> xfin(np, nullptr);
        {
            std::vector<size_t> rj;
            int smax = 0;
            for (size_t u = 0; u < np; ++u)
                if (svd_csize[u] > 0) {
                    rj.push_back(u);
                    smax = std::max(smax, ps[u]);
                }
            if (!rj.empty()) {
                std::vector<double *> X(np), Xn(np);
                for (size_t u : rj) {
                    X[u] = W + oK[u];
                    Xn[u] = W + oX2[u];
                }
                for (int it = 0; it < kRefineSteps; ++it) {
                    std::vector<GemmProb> gg, gx;
                    std::vector<RefineJob> rjobs;
                    for (size_t u : rj) {
                        const int sz = ps[u];
                        GemmProb a{};
                        a.A = X[u]; a.lda = sz; a.m = sz; a.k = sz;
                        a.B = X[u]; a.ldb = sz; a.n = sz;
                        a.C = W + oG[u]; a.ldc = sz;
                        gg.push_back(a);
                        const double tau = jobs[pending[u]].tau;
                        rjobs.push_back(RefineJob{W + oG[u], W + oIA[u], d_off + u, 0.01 * tau * tau, sz});
                        GemmProb b{};
                        b.A = X[u]; b.lda = sz; b.m = sz; b.k = sz;
                        b.B = W + oIA[u]; b.ldb = sz; b.n = sz;
                        b.C = Xn[u]; b.ldc = sz;
                        gx.push_back(b);
                    }
                    gemm_batched_small(ctx, st, true, false, gg, 1.0, 0.0);
                    TLR_CUDA_TRY(cudaMemsetAsync(d_off, 0, np * sizeof(unsigned long long), st));
                    auto *dr = (const RefineJob *)stage_push(ctx, rjobs.data(), rjobs.size() * sizeof(RefineJob), st);
                    launch(k_refine_angles, dim3((unsigned)std::min<int64_t>(ceil_div(smax * smax, 256), 64),
                                                 (unsigned)rjobs.size()), 256, 0, st, dr);
                    TLR_CHECK_LAUNCH();
                    gemm_batched_small(ctx, st, false, false, gx, 1.0, 0.0);
                    for (size_t u : rj) std::swap(X[u], Xn[u]);
                }
                std::vector<EmitJob> ej;
                for (size_t u : rj) {
                    ej.push_back(EmitJob{X[u], W + oW[u], W + oS[u], d_rank + u, d_off + u, ps[u], jobs[pending[u]].tau});
                    xfin[u] = X[u];
                }
                auto *de = (const EmitJob *)stage_push(ctx, ej.data(), ej.size() * sizeof(EmitJob), st);
                launch(k_svd_emit, (unsigned)ej.size(), kQrThreads, (size_t)smax * sizeof(double), st, de);
                TLR_CHECK_LAUNCH();
            }
        }
        cmark();
        // decisions on the host
        std::vector<int> h_rank(5 * np);
        TLR_CUDA_TRY(cudaMemcpyAsync(h_rank.data(), d_rank, 5 * np * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (overlap && !overlapped) {
            overlapped = true;
            overlap();
        }
        TLR_CUDA_TRY(cudaStreamSynchronize(st));
        stage_reset(ctx, st);
        {
            // tiles whose Gram refinement did not converge: FP64 Jacobi sweeps on the refined M1
            std::vector<SvdJob> fin;
            for (size_t u = 0; u < np; ++u)
                if (h_rank[u] == -2)
                    fin.push_back(SvdJob{W + oR[u], xfin[u], W + oW[u], W + oS[u], d_rank + u, d_rank + np + 4 * u, ps[u],
                                         jobs[pending[u]].tau});
            if (!fin.empty()) {
                std::vector<int> cs_fin;
                svd_launch(ctx, st, fin, cs_fin, nullptr, kJacFinish);
                TLR_CUDA_TRY(cudaMemcpyAsync(h_rank.data(), d_rank, 5 * np * sizeof(int), cudaMemcpyDeviceToHost, st));
                TLR_CUDA_TRY(cudaStreamSynchronize(st));
            }
        }
        cmark();
        ctx->comp_stats[0] += (long long)np;
        ctx->comp_stats[1] += 1;
        for (size_t u = 0; u < np; ++u) {
            const int *sw = h_rank.data() + np + 4 * u;
            ctx->comp_stats[2] += sw[0];
            ctx->comp_stats[3] = std::max(ctx->comp_stats[3], (long long)sw[0]);
            ctx->comp_stats[4] += sw[1];
        }
        if (ctx->profile && t16.csize == 16) {
            // FP64 work of the 16-CTA Jacobi launch, counted as executed:
            // M1 = M J (2 s^3), the norms at each FP64 sweep and at the end
            // (2 s^2 each), one dot product per pair checked (2 s), one
            // rotation of two columns per pair rotated (6 s)
            float ms = 0.f;
            TLR_CUDA_TRY(cudaEventElapsedTime(&ms, t16.e0, t16.e1));
            double fl = 0.0;
            int jobs16 = 0;
            for (size_t u = 0; u < np; ++u) {
                if (svd_csize[u] != 16) continue;
                const int *sw = h_rank.data() + np + 4 * u;
                const double s = ps[u];
                fl += 2.0 * s * s * s + 2.0 * s * s * (sw[0] + 1) + 2.0 * s * sw[2] + 6.0 * s * sw[3];
                ++jobs16;
            }
            ctx->k16_ms += ms;
            ctx->k16_flops += fl;
            ctx->k16_launches += 1;
            ctx->k16_clusters += jobs16;
        }
        std::vector<int> next;
        std::vector<GemmProb> gu, gv;
        std::vector<SplitDesc> suv;
        for (size_t u = 0; u < np; ++u) {
            int q = pending[u];
            const CompressJob &J = jobs[q];
            int s = ps[u];
            int full = std::min(J.m, J.k);
            int r = h_rank[u];
            if (r < 0) {  // non-finite singular values
                ranks[q] = kCompNan;
                fail_order.push_back(q);
                continue;
            }
            if (r > J.maxrank) {  // S are lower bounds of the tile's singular values
                ranks[q] = kCompBad;
                fail_order.push_back(q);
                continue;
            }
            double *Uo = J.U, *Vo = J.V;
            const int cap = J.cap > 0 ? J.cap : J.maxrank;
            bool conv = (s >= full) || (r <= s - kSpare);
            if (!conv) {
                if (s >= kMaxSample) {
                    ranks[q] = kCompBad;
                    fail_order.push_back(q);
                    continue;
                }
                int want = std::max(2 * s, ((r + kOversample + 7) / 8) * 8);
                sz[q] = std::min(full, std::min(want, kMaxSample));
                next.push_back(q);
                continue;
            }
            if (r > cap && !(grow && grow(J, r, &Uo, &Vo))) {
                ranks[q] = kCompBad;
                fail_order.push_back(q);
                continue;
            }
            ranks[q] = r;
            if (r == 0) continue;
            // U = Q W_r, V = B W_r (paired FP32 on the mixed paths: Q's paired
            // copy exists, B and W_r are split here)
            GemmProb a{};
            a.A = W + oQ[u]; a.lda = J.m; a.m = J.m; a.k = s;
            a.B = W + oW[u]; a.ldb = s; a.n = r;
            a.C = Uo; a.ldc = J.ldu;
            GemmProb b{};
            b.A = W + oB[u]; b.lda = J.k; b.m = J.k; b.k = s;
            b.B = W + oW[u]; b.ldb = s; b.n = r;
            b.C = Vo; b.ldc = J.ldv;
            if (dfp) {
                float2 *b2 = (float2 *)(W + oB2[u]), *w2 = (float2 *)(W + oW2[u]);
                suv.push_back(SplitDesc{W + oB[u], b2, J.k, J.k, s});
                suv.push_back(SplitDesc{W + oW[u], w2, s, s, r});
                a.A2 = (const float2 *)(W + oQ2[u]);
                a.B2 = w2;
                b.A2 = b2;
                b.B2 = w2;
            }
            gu.push_back(a);
            gv.push_back(b);
        }
        split_f2_batched(ctx, st, suv);
        gemm_batched(ctx, st, false, false, gu, 1.0, 0.0, dfp);
        gemm_batched(ctx, st, false, false, gv, 1.0, 0.0, dfp);
        cmark();
        // the workspace is released stream-ordered after these GEMMs
        pending.swap(next);
    }
    if (overlap && !overlapped) overlap();  // nothing was compressed
}

void compress_profile_reset(tlr_ctx *ctx) {
    ctx->comp_pending.clear();
    ctx->comp_used = 0;
}

void compress_profile_collect(tlr_ctx *ctx) {
    const std::vector<cudaEvent_t> &ev = ctx->comp_pending;
    for (size_t c = 0; c + 8 <= ev.size(); c += 8) {
        TLR_CUDA_TRY(cudaEventSynchronize(ev[c + 7]));
        for (int k = 0; k < 7; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[c + k], ev[c + k + 1]) == cudaSuccess) ctx->comp_ms[k] += ms;
        }
    }
    compress_profile_reset(ctx);
}

void compress_tiles(tlr_ctx *ctx, cudaStream_t st, std::vector<CompressJob> &jobs, double tau, int maxrank,
                    std::vector<int> &ranks, long long *bad_tile, long long *nan_tile, bool df,
                    const std::function<void()> &overlap, const GrowSlot &grow, bool tc) {
    for (CompressJob &J : jobs) {
        J.tau = tau;
        J.maxrank = maxrank;
    }
    std::vector<int> fails;
    compress_profile_reset(ctx);
    compress_jobs(ctx, st, jobs, ranks, fails, df, overlap, grow, tc);
    if (ctx->profile) compress_profile_collect(ctx);
    *bad_tile = *nan_tile = -1;
    for (int q : fails) {
        long long *first = ranks[(size_t)q] == kCompNan ? nan_tile : bad_tile;
        if (*first < 0) *first = jobs[(size_t)q].tile_id;
        ranks[(size_t)q] = 0;
    }
}

}  // namespace tlr

// Device Matern covariance (Eq. 4.2) with a device K_nu.
//
//   C(d) = sigma2 * 2^(1-nu) / Gamma(nu) * x^nu * K_nu(x),  x = d / beta,  C(0) = sigma2.
//
// K_nu for real nu > 0: write nu = mu + m with m = floor(nu + 1/2) and
// mu in [-1/2, 1/2); compute K_mu and K_{mu+1}, then recur upward with
// K_{a+1} = K_{a-1} + (2a/x) K_a (stable for K in increasing order).
//
//  x <= 2:       Temme's series (N. M. Temme, J. Comput. Phys. 19 (1975) 324):
//                K_mu = sum c_k f_k, K_{mu+1} = (2/x) sum c_k (p_k - k f_k), with
//                c_k = (x^2/4)^k / k!, f_0 from Gamma1/Gamma2, p_0 = (x/2)^-mu Gamma(1+mu)/2,
//                q_0 = (x/2)^mu Gamma(1-mu)/2, f_k = (k f_{k-1} + p_{k-1} + q_{k-1})/(k^2-mu^2),
//                p_k = p_{k-1}/(k-mu), q_k = q_{k-1}/(k+mu).
//  2 < x <= 25:  K_mu(x) = sqrt(pi) (2x)^mu e^-x U(mu+1/2, 2mu+1, 2x) (DLMF 10.39.6).  The
//                sequence u_k = U(mu+1/2+k, 2mu+1, 2x) obeys
//                u_{k-1} - 2(k+x) u_k + ((k+1/2)^2 - mu^2) u_{k+1} = 0 (DLMF 13.3.7) and
//                is its minimal solution, so h = u_1/u_0 is a continued fraction
//                evaluated backwards; then K_{mu+1}/K_mu = (mu + 1/2 + x + (mu^2 - 1/4) h)/x,
//                and the Wronskian I_mu K_{mu+1} + I_{mu+1} K_mu = 1/x (DLMF 10.28.2)
//                with the (positive-term) power series of I fixes the scale.
//  x > 25:       the asymptotic expansion e^x K_mu(x) ~ sqrt(pi/2x) sum_k a_k(mu) x^-k,
//                a_k = a_{k-1} (4mu^2 - (2k-1)^2) / (8k); its smallest term is below e^-2x.
//
// All per-theta constants (Gamma values, series denominators) are computed
// once on the host (MaternParams) so the per-entry work is multiplies/adds,
// one log, one or two exps and a few divisions.
#pragma once

#include <cuda_runtime.h>

namespace tlr {

constexpr int kTemmeTerms = 22;   // (x^2/4)^k / k! < 1e-21 at x = 2
constexpr int kISeriesTerms = 64; // I-series terms for x <= 25
constexpr int kAsymTerms = 30;    // asymptotic terms for x > 25

// Per-theta interpolation table of log C(d)/sigma2 as a function of s = d^2:
// each binade [2^e, 2^(e+1)) of s (kTabEmin <= e <= kTabEmax) is split into
// kTabSub equal sub-intervals, and on each the function is replaced by its
// degree-kTabDeg Chebyshev interpolant.  log C is analytic on each interval
// (its only singularity is s = 0), so the interpolants converge
// geometrically; with these sizes the error is below 1e-13 relative.  An
// interval whose nodes underflow is flagged (c_0 = NaN) and evaluated
// directly.
constexpr int kTabEmin = -44, kTabEmax = 3, kTabSub = 4, kTabDeg = 12;
constexpr int kTabIntervals = (kTabEmax - kTabEmin + 1) * kTabSub;
constexpr int kTabCoef = kTabDeg + 1;

struct MaternParams {
    double sigma2, inv_beta, nu;
    const double *tab;  // kTabIntervals x kTabCoef Chebyshev coefficients, or null (direct K_nu)
    const float2 *tab2; // the same coefficients as (hi, lo) FP32 pairs (paired-FP32 evaluation), or null
    double mu;
    int m;
    double lead;       // 2^(1-nu) / Gamma(nu)
    double g1, g2;     // Temme's Gamma1(mu), Gamma2(mu)
    double gp, gm;     // Gamma(1+mu), Gamma(1-mu)
    double mupi_sin;   // mu pi / sin(mu pi)
    double inv_gmu1;   // 1 / Gamma(mu+1)
    double inv_gmu2;   // 1 / Gamma(mu+2)
    double tf[kTemmeTerms + 1];  // 1/(k^2 - mu^2)
    double tp[kTemmeTerms + 1];  // 1/(k - mu)
    double tq[kTemmeTerms + 1];  // 1/(k + mu)
    double tk[kTemmeTerms + 1];  // 1/k
    double ti0[kISeriesTerms + 1];  // 1/(k (k + mu))
    double ti1[kISeriesTerms + 1];  // 1/(k (k + mu + 1))
    double ta0[kAsymTerms + 1];     // (4mu^2 - (2k-1)^2) / (8k)
    double ta1[kAsymTerms + 1];     // same for mu + 1
};

// Returns K_mu and K_{mu+1}; *scaled = true when both are multiplied by e^x.
__device__ __forceinline__ void bessel_k_pair(double x, const MaternParams &P, double &k0,
                                              double &k1, bool &scaled) {
    const double mu = P.mu;
    if (x <= 2.0) {
        double l2x = log(2.0 / x);
        double sg = mu * l2x;
        double es = exp(sg), ies = 1.0 / es;
        double chs = 0.5 * (es + ies);
        double shs_s;
        if (fabs(sg) < 1e-3) {
            double s2 = sg * sg;
            shs_s = 1.0 + s2 * (1.0 / 6.0 + s2 * (1.0 / 120.0));
        } else {
            shs_s = 0.5 * (es - ies) / sg;
        }
        double f = P.mupi_sin * (chs * P.g1 + shs_s * l2x * P.g2);
        double p = 0.5 * es * P.gp;
        double q = 0.5 * ies * P.gm;
        double c = 1.0;
        double x2 = 0.25 * x * x;
        double s0 = f, s1 = p;
#pragma unroll 2
        for (int k = 1; k <= kTemmeTerms; ++k) {
            f = ((double)k * f + p + q) * P.tf[k];
            p *= P.tp[k];
            q *= P.tq[k];
            c *= x2 * P.tk[k];
            s0 += c * f;
            s1 += c * (p - (double)k * f);
        }
        k0 = s0;
        k1 = s1 * (2.0 / x);
        scaled = false;
        return;
    }
    if (x <= 25.0) {
        // continued fraction for h = u_1 / u_0, evaluated from depth K down to 1
        double sq = sqrt(2.0 * x);
        int K = (int)((10.0 + sq) * (10.0 + sq) / (2.0 * x)) + 6;
        double mu2 = mu * mu;
        double t = 0.0;
        for (int k = K; k >= 1; --k) {
            double kh = (double)k + 0.5;
            t = 1.0 / (2.0 * ((double)k + x) - (kh * kh - mu2) * t);
        }
        double rho = (mu + 0.5 + x + (mu2 - 0.25) * t) / x;  // K_{mu+1} / K_mu
        // e^-x I_mu and e^-x I_{mu+1} from their power series
        double x2 = 0.25 * x * x;
        double a0 = 1.0, a1 = 1.0, s0 = 1.0, s1 = 1.0;
        for (int k = 1; k <= kISeriesTerms; ++k) {
            a0 *= x2 * P.ti0[k];
            a1 *= x2 * P.ti1[k];
            s0 += a0;
            s1 += a1;
        }
        double pre = exp(mu * log(0.5 * x) - x);  // (x/2)^mu e^-x
        double i0 = pre * P.inv_gmu1 * s0;
        double i1 = pre * (0.5 * x) * P.inv_gmu2 * s1;
        k0 = 1.0 / (x * (rho * i0 + i1));
        k1 = rho * k0;
        scaled = true;
        return;
    }
    {
        double ix = 1.0 / x;
        double a0 = 1.0, a1 = 1.0, s0 = 1.0, s1 = 1.0;
        for (int k = 1; k <= kAsymTerms; ++k) {
            a0 *= P.ta0[k] * ix;
            a1 *= P.ta1[k] * ix;
            s0 += a0;
            s1 += a1;
        }
        double pre = sqrt(1.5707963267948966 * ix);  // sqrt(pi / 2x)
        k0 = pre * s0;
        k1 = pre * s1;
        scaled = true;
    }
}

// C(d) / sigma2 for d > 0 given x = d / beta.
__device__ __forceinline__ double matern_corr_x(double x, const MaternParams &P) {
    double k0, k1;
    bool scaled;
    bessel_k_pair(x, P, k0, k1, scaled);
    double kn;
    if (P.m == 0) {
        kn = k0;
    } else {
        double a = k0, b = k1, tix = 2.0 / x;
        for (int k = 1; k < P.m; ++k) {
            double c = a + (P.mu + (double)k) * tix * b;
            a = b;
            b = c;
        }
        kn = b;
    }
    double lx = log(x);
    return P.lead * exp(P.nu * lx - (scaled ? x : 0.0)) * kn;
}

// C(d)/sigma2 from the squared distance s > 0 through the table (falls back to
// the direct K_nu outside the table or on flagged intervals).
__device__ __forceinline__ double matern_corr_s(double s, const MaternParams &P) {
    if (P.tab) {
        long long bits = __double_as_longlong(s);
        int e = (int)((bits >> 52) & 0x7FF) - 1023;
        if (e >= kTabEmin && e <= kTabEmax) {
            int sub = (int)((bits >> 50) & 3);
            // fraction of the binade in [0, 1), exact
            double u = (double)(bits & 0xFFFFFFFFFFFFFll) * 2.220446049250313e-16;
            double t = 2.0 * (u * kTabSub - (double)sub) - 1.0;
            const double *c = P.tab + ((e - kTabEmin) * kTabSub + sub) * kTabCoef;
            double c0 = __ldg(c);
            if (c0 == c0) {
                double b1 = 0.0, b2 = 0.0, t2 = 2.0 * t;
#pragma unroll
                for (int j = kTabDeg; j >= 1; --j) {
                    double b0 = fma(t2, b1, __ldg(c + j) - b2);
                    b2 = b1;
                    b1 = b0;
                }
                return exp(fma(t, b1, c0 - b2));
            }
        }
    }
    return matern_corr_x(sqrt(s) * P.inv_beta, P);
}

// Covariance between two locations.
__device__ __forceinline__ double matern_cov(double xa, double ya, double xb, double yb,
                                             const MaternParams &P) {
    double dx = xa - xb, dy = ya - yb;
    double s = dx * dx + dy * dy;
    if (s == 0.0) return P.sigma2;
    return P.sigma2 * matern_corr_s(s, P);
}

// ---- the table in paired FP32 ("float-float", Dekker 1971): the same
// Chebyshev interpolant of log C, evaluated with ~47-bit FP32 pairs on the
// FP32 pipe (64 times GB300's FP64 rate), then exp in the same arithmetic.
// Used by the covariance panels of the mixed-precision paths; the FP64 path
// keeps matern_cov.
struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.h, b.h);
    return ff_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_fast(p, e);
}

// exp(y) for y <= ~0 in paired FP32: y = k ln2 + r with ln2 in three parts
// (the first of 16 bits, so that k times it is exact for |k| < 2^8), then the
// Taylor polynomial of exp(r), |r| <= ln2 / 2, to degree 12 (truncation below
// 2^-47): degrees 7-12 in FP32 on r's high word, 0-6 in pairs.  Below -87
// (under FP32's normal range) the result is 0.
__device__ __forceinline__ FF ff_exp(FF y) {
    if (y.h < -87.0f) return FF{0.f, 0.f};
    const float k = rintf(__fmul_rn(y.h, 1.44269504f));
    const float L1 = 0.693145751953125f, L2 = 1.428606765330187e-06f, L3 = 5.495603971894525e-14f;
    FF r = ff_fast(__fsub_rn(y.h, __fmul_rn(k, L1)), y.l);       // y - k L1 (exact first word)
    const float p2 = __fmul_rn(k, L2), p2e = __fmaf_rn(k, L2, -p2);  // k L2 exactly, as a pair
    r = ff_add(r, FF{-p2, -p2e});
    r = ff_add(r, FF{__fmul_rn(-k, L3), 0.f});
    const float rh = r.h;
    float q = 2.0876756e-09f;  // 1/12!
    q = __fmaf_rn(q, rh, 2.5052108e-08f);
    q = __fmaf_rn(q, rh, 2.755732e-07f);
    q = __fmaf_rn(q, rh, 2.7557319e-06f);
    q = __fmaf_rn(q, rh, 2.4801588e-05f);
    q = __fmaf_rn(q, rh, 1.984127e-04f);  // ... + 1/7! (high word)
    FF e{q, 0.f};
    const FF c[7] = {FF{1.0f, 0.f}, FF{1.0f, 0.f}, FF{0.5f, 0.f}, FF{0.16666667f, -4.967054e-09f},
                     FF{0.041666668f, -1.2417635e-09f}, FF{0.008333334f, -4.346172e-10f},
                     FF{0.0013888889f, -3.3631094e-11f}};
    e = ff_add(FF{-2.7255969e-12f, 0.f}, e);  // 1/7! low word
#pragma unroll
    for (int j = 6; j >= 0; --j) e = ff_add(c[j], ff_mul(r, e));
    const int ki = (int)k;
    return FF{ldexpf(e.h, ki), ldexpf(e.l, ki)};
}

// C(d)/sigma2 from s = d^2 through the paired-FP32 table; false (nothing
// written) outside the table or on a flagged interval.
__device__ __forceinline__ bool matern_corr_s_ff(double s, const MaternParams &P, double *out) {
    if (!P.tab2) return false;
    const long long bits = __double_as_longlong(s);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;
    if (e < kTabEmin || e > kTabEmax) return false;
    const int sub = (int)((bits >> 50) & 3);
    // t = 2 frac(4 u) - 1 from the 50 fraction bits below the two sub-interval bits
    const long long f = bits & 0x3FFFFFFFFFFFFll;
    const float th = __fsub_rn(__fmul_rn((float)(int)(f >> 26), 1.1920928955078125e-07f), 1.0f);  // 2^-23
    const float tl = __fmul_rn((float)(int)(f & 0x3FFFFFFll), 1.7763568394002505e-15f);          // 2^-49
    const FF t = ff_fast(th, tl);
    const FF t2{__fmul_rn(2.0f, t.h), __fmul_rn(2.0f, t.l)};
    const float2 *c = P.tab2 + ((e - kTabEmin) * kTabSub + sub) * kTabCoef;
    const float2 c0 = __ldg(c);
    if (c0.x != c0.x) return false;
    FF b1{0.f, 0.f}, b2{0.f, 0.f};
#pragma unroll
    for (int j = kTabDeg; j >= 1; --j) {
        const float2 cj = __ldg(c + j);
        const FF b0 = ff_add(ff_add(FF{cj.x, cj.y}, ff_mul(t2, b1)), FF{-b2.h, -b2.l});
        b2 = b1;
        b1 = b0;
    }
    const FF lg = ff_add(ff_add(FF{c0.x, c0.y}, ff_mul(t, b1)), FF{-b2.h, -b2.l});
    const FF ex = ff_exp(lg);
    *out = (double)ex.h + (double)ex.l;
    return true;
}

// Covariance between two locations, the table evaluated in paired FP32
// (~1e-14 relative; matern_cov outside the table).
__device__ __forceinline__ double matern_cov_ff(double xa, double ya, double xb, double yb,
                                                const MaternParams &P) {
    const double dx = xa - xb, dy = ya - yb;
    const double s = dx * dx + dy * dy;
    if (s == 0.0) return P.sigma2;
    double c;
    if (matern_corr_s_ff(s, P, &c)) return P.sigma2 * c;
    return P.sigma2 * matern_corr_s(s, P);
}

// Host: per-theta constants.  Returns false if theta is not positive/finite.
// The table pointer is left null (direct K_nu).
bool make_matern_params(double sigma2, double beta, double nu, MaternParams *out);

// Build the interpolation table of P into `tab` (kTabIntervals * kTabCoef
// doubles, device) on stream s and point P->tab at it.
void build_matern_table(MaternParams *P, double *tab, cudaStream_t s);

}  // namespace tlr

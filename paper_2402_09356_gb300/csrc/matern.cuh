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

// Host: per-theta constants.  Returns false if theta is not positive/finite.
// The table pointer is left null (direct K_nu).
bool make_matern_params(double sigma2, double beta, double nu, MaternParams *out);

// Build the interpolation table of P into `tab` (kTabIntervals * kTabCoef
// doubles, device) on stream s and point P->tab at it.
void build_matern_table(MaternParams *P, double *tab, cudaStream_t s);

}  // namespace tlr

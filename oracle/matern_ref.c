/*
 * CPU FP64 oracle, part 1 of 2: the modified Bessel function of the second
 * kind K_nu and the Matern covariance of Eq. 4.2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/_liboracle.so
 * and is loaded only by tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py.  It shares no code with the CUDA path.
 *
 * K_nu (Sec. 4.1, below Eq. 4.2): for x > 0 and real nu,
 *     K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 * (the standard integral representation, e.g. DLMF 10.32.9).  We write
 *     K_nu(x) = exp(-x) * int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt
 * and evaluate the integral with the trapezoid rule on a uniform grid of step
 * h.  The integrand is even in t and analytic in a strip around the real
 * axis, so the rule (half weight at t = 0) converges geometrically in 1/h;
 * near the peak the integrand behaves like exp(-x t^2 / 2), whose trapezoid
 * error is about 2 exp(-2 pi^2 / (x h^2)), hence h = min(0.1, 0.5/sqrt(x))
 * (error below 1e-17 for every x).  All terms are positive: no cancellation.
 * cosh t - 1 is computed as 2 sinh^2(t/2) to keep relative accuracy near 0.
 *
 * Matern covariance (Eq. 4.2): with x = d / beta,
 *     C(d) = sigma2 / (Gamma(nu) 2^(nu-1)) * x^nu * K_nu(x),   C(0) = sigma2.
 * x^nu exp(-x) is formed as exp(nu log x - x) so that neither factor
 * overflows on its own.
 */
#include <math.h>
#include <stdint.h>

/* Scaled integral S(nu, x) = exp(x) K_nu(x). */
static double scaled_kv_integral(double nu, double x)
{
    double h = 0.1;
    double hs = 0.5 / sqrt(x);
    if (hs < h) h = hs;
    double sum = 0.5; /* t = 0: exp(0) * cosh(0), half weight */
    for (long k = 1; k < 2000000; ++k) {
        double t = (double)k * h;
        double s = sinh(0.5 * t);
        double term = exp(-x * 2.0 * s * s) * cosh(nu * t);
        sum += term;
        /* past the peak (d/dt of the log-integrand < 0) and negligible */
        if (x * sinh(t) > fabs(nu) && term < 1e-18 * sum) break;
    }
    return h * sum;
}

double oracle_besselk(double nu, double x)
{
    if (!(x > 0.0)) return INFINITY;
    return exp(-x) * scaled_kv_integral(nu, x);
}

double oracle_besselk_scaled(double nu, double x)
{
    if (!(x > 0.0)) return INFINITY;
    return scaled_kv_integral(nu, x);
}

double oracle_matern(double d, double sigma2, double beta, double nu)
{
    if (d == 0.0) return sigma2;
    double x = d / beta;
    double lead = sigma2 / (tgamma(nu) * pow(2.0, nu - 1.0));
    return lead * exp(nu * log(x) - x) * scaled_kv_integral(nu, x);
}

/* Matern covariance for m distances. */
void oracle_matern_vec(int64_t m, const double *d, double sigma2, double beta,
                       double nu, double *out)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < m; ++k)
        out[k] = oracle_matern(d[k], sigma2, beta, nu);
}

/*
 * Dense covariance (Eq. 1.1): out[i*n + j] = C(||s_i - s_j||) for locations
 * given as SoA xy (x then y, n each).  The lower triangle is computed and
 * mirrored, so out is exactly symmetric.
 */
void oracle_matern_matrix(int64_t n, const double *xy, double sigma2, double beta,
                          double nu, double *out)
{
    const double *x = xy, *y = xy + n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double dx = x[i] - x[j];
            double dy = y[i] - y[j];
            double d = sqrt(dx * dx + dy * dy);
            double c = oracle_matern(d, sigma2, beta, nu);
            out[i * n + j] = c;
            out[j * n + i] = c;
        }
    }
}

/*
 * Rectangular block of the covariance: out[a*nc + b] = C(||s_ra - s_cb||)
 * between row locations (SoA, nr each) and column locations (SoA, nc each).
 */
void oracle_matern_block(int64_t nr, const double *rxy, int64_t nc, const double *cxy,
                         double sigma2, double beta, double nu, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nr; ++a) {
        for (int64_t b = 0; b < nc; ++b) {
            double dx = rxy[a] - cxy[b];
            double dy = rxy[nr + a] - cxy[nc + b];
            out[a * nc + b] = oracle_matern(sqrt(dx * dx + dy * dy), sigma2, beta, nu);
        }
    }
}

// a2: Matern covariance tiles (Eq. 1.1, Eq. 4.2) and the per-theta constants
// of the device K_nu.
#include <cmath>

#include "common.cuh"
#include "matern.cuh"

namespace tlr {

// zeta(k), k >= 2, by a direct sum plus the Euler-Maclaurin tail (long double).
static long double zeta_ld(int k) {
    const int N = 1000;
    long double s = 0.0L;
    for (int n = N - 1; n >= 1; --n) s += powl((long double)n, -(long double)k);
    long double Nl = N;
    s += powl(Nl, 1.0L - k) / (k - 1) + 0.5L * powl(Nl, -(long double)k) +
         (long double)k / 12.0L * powl(Nl, -(long double)k - 1.0L) -
         (long double)k * (k + 1) * (k + 2) / 720.0L * powl(Nl, -(long double)k - 3.0L);
    return s;
}

// Temme's Gamma1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu) and
// Gamma2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2 for |mu| <= 1/2.
// For small |mu| the difference cancels, so there both come from
// ln Gamma(1+z) = -gamma z + sum_{k>=2} (-1)^k zeta(k) z^k / k: with
// E = -sum_{k even} zeta(k) mu^k / k and O = gamma mu + sum_{k odd>=3} zeta(k) mu^k / k,
// 1/Gamma(1 -+ mu) = e^E e^(-+O), so Gamma1 = -e^E sinh(O)/mu and Gamma2 = e^E cosh(O).
static void temme_gammas(double mu, double *g1, double *g2) {
    long double m = mu;
    if (fabsl(m) >= 0.2L) {
        long double a = 1.0L / tgammal(1.0L - m), b = 1.0L / tgammal(1.0L + m);
        *g1 = (double)((a - b) / (2.0L * m));
        *g2 = (double)((a + b) / 2.0L);
        return;
    }
    const long double euler = 0.57721566490153286060651209008240243L;
    long double E = 0.0L, Om = euler;  // Om = O / mu
    long double prev = m;              // mu^(k-1)
    for (int k = 2; k <= 40; ++k) {
        long double cur = prev * m;    // mu^k
        long double z = zeta_ld(k);
        if (k % 2 == 0) E -= z * cur / k;
        else Om += z * prev / k;
        prev = cur;
    }
    long double O = Om * m;
    long double shr = (fabsl(O) < 1e-12L) ? 1.0L + O * O / 6.0L : sinhl(O) / O;  // sinh(O)/O
    *g1 = (double)(-expl(E) * shr * Om);
    *g2 = (double)(expl(E) * coshl(O));
}

bool make_matern_params(double sigma2, double beta, double nu, MaternParams *P) {
    if (!(sigma2 > 0) || !(beta > 0) || !(nu > 0) || !std::isfinite(sigma2) || !std::isfinite(beta) ||
        !std::isfinite(nu) || nu > 50.0)
        return false;
    P->sigma2 = sigma2;
    P->inv_beta = 1.0 / beta;
    P->tab = nullptr;
    P->nu = nu;
    int m = (int)std::floor(nu + 0.5);
    double mu = nu - m;
    P->m = m;
    P->mu = mu;
    P->lead = (double)(powl(2.0L, 1.0L - (long double)nu) / tgammal((long double)nu));
    temme_gammas(mu, &P->g1, &P->g2);
    P->gp = (double)tgammal(1.0L + (long double)mu);
    P->gm = (double)tgammal(1.0L - (long double)mu);
    long double mpi = (long double)mu * 3.14159265358979323846264338327950288L;
    P->mupi_sin = (fabsl(mpi) < 1e-6L) ? (double)(1.0L + mpi * mpi / 6.0L) : (double)(mpi / sinl(mpi));
    P->inv_gmu1 = (double)(1.0L / tgammal((long double)mu + 1.0L));
    P->inv_gmu2 = (double)(1.0L / tgammal((long double)mu + 2.0L));
    for (int k = 0; k <= kTemmeTerms; ++k) {
        long double kk = k;
        P->tf[k] = k ? (double)(1.0L / (kk * kk - (long double)mu * mu)) : 0.0;
        P->tp[k] = k ? (double)(1.0L / (kk - mu)) : 0.0;
        P->tq[k] = k ? (double)(1.0L / (kk + mu)) : 0.0;
        P->tk[k] = k ? (double)(1.0L / kk) : 0.0;
    }
    for (int k = 0; k <= kISeriesTerms; ++k) {
        long double kk = k;
        P->ti0[k] = k ? (double)(1.0L / (kk * (kk + mu))) : 0.0;
        P->ti1[k] = k ? (double)(1.0L / (kk * (kk + mu + 1.0L))) : 0.0;
    }
    for (int k = 0; k <= kAsymTerms; ++k) {
        long double kk = k, a = 4.0L * mu * mu, b = 4.0L * (mu + 1.0L) * (mu + 1.0L);
        long double o = (2.0L * kk - 1.0L) * (2.0L * kk - 1.0L);
        P->ta0[k] = k ? (double)((a - o) / (8.0L * kk)) : 0.0;
        P->ta1[k] = k ? (double)((b - o) / (8.0L * kk)) : 0.0;
    }
    return true;
}

// Packed lower-triangular tiles: blockIdx.y = packed tile index, each block
// fills a 32 x 32 sub-block; threads run down the columns (coalesced stores).
__global__ void k_generate_tiles(const double *__restrict__ xy, int64_t n, int nb, int nt,
                                 MaternParams P, double *__restrict__ tiles) {
    int sub = nb / 32 + (nb % 32 != 0);
    int64_t t = (int64_t)blockIdx.x / (sub * sub);
    int sb = (int)((int64_t)blockIdx.x % (sub * sub));
    // tile (i, j) from packed index t = i (i + 1) / 2 + j
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
    while ((int64_t)i * (i + 1) / 2 > t) --i;
    int j = (int)(t - (int64_t)i * (i + 1) / 2);
    int br = sb % sub, bc = sb / sub;
    int r = br * 32 + (threadIdx.x & 31);
    int c0 = bc * 32 + (threadIdx.x >> 5) * 4;
    int64_t gr = (int64_t)i * nb + r;
    double *T = tiles + t * (int64_t)nb * nb;
    bool rv = r < nb && gr < n;
    double xr = rv ? xy[gr] : 0.0, yr = rv ? xy[n + gr] : 0.0;
    for (int q = 0; q < 4; ++q) {
        int c = c0 + q;
        if (c >= nb || r >= nb) continue;
        int64_t gc = (int64_t)j * nb + c;
        double v = 0.0;
        if (rv && gc < n) v = matern_cov(xr, yr, xy[gc], xy[n + gc], P);
        T[(int64_t)c * nb + r] = v;
    }
    (void)nt;
}

// A column panel of the covariance: T[c * ld + r] = C(s_{ri0 + r}, s_{ci0 + c})
// for r < rows, c < cols; rows or columns past n give 0.  Each block fills a
// 32-row x 32-column sub-block, threads down the columns (coalesced stores).
__global__ void k_generate_panel(const double *__restrict__ xy, int64_t n, int64_t ri0, int64_t ci0, int rows,
                                 int cols, MaternParams P, double *__restrict__ T, int ld) {
    const int r = blockIdx.x * 32 + (threadIdx.x & 31);
    const int c0 = blockIdx.y * 32 + (threadIdx.x >> 5) * 4;
    if (r >= rows) return;
    const int64_t gr = ri0 + r;
    const bool rv = gr < n;
    const double xr = rv ? xy[gr] : 0.0, yr = rv ? xy[n + gr] : 0.0;
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + q;
        if (c >= cols) break;
        const int64_t gc = ci0 + c;
        T[(int64_t)c * ld + r] = (rv && gc < n) ? matern_cov(xr, yr, xy[gc], xy[n + gc], P) : 0.0;
    }
}

__global__ void k_matern_vec(const double *__restrict__ d, int64_t m, MaternParams P,
                             double *__restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double v = d[k];
    if (v == 0.0) out[k] = P.sigma2;
    else if (P.tab) out[k] = P.sigma2 * matern_corr_s(v * v, P);
    else out[k] = P.sigma2 * matern_corr_x(v * P.inv_beta, P);
}

// Table nodes: log C/sigma2 at the Chebyshev points of every interval.
__global__ void k_table_nodes(MaternParams P, double *__restrict__ g) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kTabIntervals * kTabCoef) return;
    int iv = q / kTabCoef, k = q % kTabCoef;
    int e = kTabEmin + iv / kTabSub, sub = iv % kTabSub;
    double lo = ldexp(1.0 + (double)sub / kTabSub, e), hi = ldexp(1.0 + (double)(sub + 1) / kTabSub, e);
    double node = cospi((k + 0.5) / kTabCoef);
    double sv = lo + 0.5 * (node + 1.0) * (hi - lo);
    double c = matern_corr_x(sqrt(sv) * P.inv_beta, P);
    g[q] = (c > 1e-280) ? log(c) : __longlong_as_double(0x7FF8000000000000ll);
}

// Chebyshev coefficients c_j = (2/N) sum_k g_k cos(j pi (k + 1/2) / N), c_0 halved;
// an interval with a non-finite node value keeps c_0 = NaN (direct evaluation).
__global__ void k_table_coefs(const double *__restrict__ g, double *__restrict__ tab) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kTabIntervals * kTabCoef) return;
    int iv = q / kTabCoef, j = q % kTabCoef;
    const double *gi = g + iv * kTabCoef;
    double acc = 0.0;
    bool bad = false;
    for (int k = 0; k < kTabCoef; ++k) {
        double v = gi[k];
        bad |= !(v == v);
        acc += v * cospi((double)j * (k + 0.5) / kTabCoef);
    }
    acc *= 2.0 / kTabCoef;
    if (j == 0) acc *= 0.5;
    if (bad && j == 0) acc = __longlong_as_double(0x7FF8000000000000ll);
    tab[q] = acc;
}

void build_matern_table(MaternParams *P, double *tab, cudaStream_t s) {
    const int cnt = kTabIntervals * kTabCoef;
    double *g = tab + cnt;  // scratch: the caller provides 2 * cnt doubles
    MaternParams direct = *P;
    direct.tab = nullptr;
    launch(k_table_nodes, (unsigned)ceil_div(cnt, 128), 128, 0, s, direct, g);
    launch(k_table_coefs, (unsigned)ceil_div(cnt, 128), 128, 0, s, g, tab);
    TLR_CHECK_LAUNCH();
    P->tab = tab;
}

void generate_tiles(const double *xy, int64_t n, int nb, const MaternParams &P, double *tiles,
                    cudaStream_t s) {
    int nt = (int)ceil_div(n, nb);
    int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
    int sub = (int)ceil_div(nb, 32);
    launch(k_generate_tiles, (unsigned)(ntiles * sub * sub), 256, 0, s, xy, n, nb, nt, P, tiles);
    TLR_CHECK_LAUNCH();
}

void generate_panel(const double *xy, int64_t n, int64_t ri0, int64_t ci0, int rows, int cols,
                    const MaternParams &P, double *T, int ld, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    launch(k_generate_panel, dim3((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32)), 256, 0, s, xy, n, ri0,
           ci0, rows, cols, P, T, ld);
    TLR_CHECK_LAUNCH();
}

void matern_vec(const double *d, int64_t m, const MaternParams &P, double *out, cudaStream_t s) {
    if (m > 0) launch(k_matern_vec, (unsigned)ceil_div(m, 256), 256, 0, s, d, m, P, out);
    TLR_CHECK_LAUNCH();
}

}  // namespace tlr

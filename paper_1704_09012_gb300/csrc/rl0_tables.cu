// rl0_tables.cu -- host-side constants of a decode, in FP64 (arXiv 1704.09012):
// the Gaussian posterior series of Eqs. (pz_approx)/(pe_approx) normalised per
// Eq. (breve), the sweep step of Eqs. (finetune_c_quant)/(finetune_c_cont), and
// the per-round magnitude thresholds that turn the score tests of Table
// "scores" into exact comparisons on FP32 values.  One function computes them
// for every entry point, so the single-instance and batched decoders use the
// same constants bit for bit.
#include <cmath>
#include <cstring>

#include "rl0_common.cuh"

namespace rl0 {

// Eq. (pz_approx) (lam = d rho, vn = s_n^2) or Eq. (pe_approx) (lam = 2 d rho,
// vn = 2 s_n^2): terms q = 0..ell with weight lam^q/q! and variance
// q s_s^2 + vn, and the tail R(ell) = sum_{q>ell} lam^q/q! with the
// variance-matched v = (s_s^2 lam R(ell-1) + vn R(ell)) / R(ell).  Dividing
// numerator and denominator by the noise density gives
//   p(0)/p(w) = sum_terms c_t sqrt(vn/v_t) exp(w^2 (1/(2 vn) - 1/(2 v_t))) / D,
// with D the same sum at w = 0 (the maximum of p is at 0).
HostSeries make_series(double lam, double s2, double vn, int ell)
{
    double wt[RL0_MAXQ], var[RL0_MAXQ];
    int nt = 0;
    double term = 1.0;
    for (int q = 0; q <= ell; ++q) {
        if (q > 0) term *= lam / q;
        wt[nt] = term;
        var[nt] = q * s2 + vn;
        ++nt;
    }
    // tails R(ell) and R(ell - 1), summed directly
    double tq = term, Rl = 0.0;
    for (int q = ell + 1; q < ell + 4000; ++q) {
        tq *= lam / q;
        Rl += tq;
        if (tq == 0.0 || (q > lam && tq < Rl * 1e-18)) break;
    }
    const double Rlm1 = Rl + term;               // adds the q = ell term
    if (Rl > 0.0) {
        wt[nt] = Rl;
        var[nt] = (s2 * lam * Rlm1 + vn * Rl) / Rl;
        ++nt;
    }
    HostSeries H;
    std::memset(&H, 0, sizeof(H));
    H.nq = nt;
    double D = 0.0;
    for (int q = 0; q < nt; ++q) D += wt[q] * std::sqrt(vn / var[q]);
    for (int q = 0; q < nt; ++q) {
        H.a[q] = wt[q] * std::sqrt(vn / var[q]) / D;
        H.b[q] = 0.5 / vn - 0.5 / var[q];
    }
    H.b[0] = 0.0;
    return H;
}

// F(w) = p_breve(w)^-1 = sum_q a_q exp(b_q w^2).
double series_F(const HostSeries &H, double w)
{
    const double u = w * w;
    double acc = 0.0;
    for (int q = 0; q < H.nq; ++q) acc += H.a[q] * std::exp(H.b[q] * u);
    return acc;
}

// Root w >= 0 of F(w) = T for T > 1.  In u = w^2, F is a positive sum of
// exponentials: increasing and convex, so Newton's method started above the
// root decreases monotonically onto it.  The start comes from the bracket
// a_0 + A exp(b_min u) <= F <= a_0 + A exp(b_max u), A = sum_{q>=1} a_q.
static double series_root(const HostSeries &H, double T)
{
    double bmin = INFINITY, A = 0.0;
    for (int q = 1; q < H.nq; ++q) { bmin = std::fmin(bmin, H.b[q]); A += H.a[q]; }
    const double L = std::log((T - H.a[0]) / A);
    double u = (L > 0.0 && bmin > 0.0) ? 1.0001 * L / bmin : 1.0;
    while (series_F(H, std::sqrt(u)) < T) u *= 2.0;
    for (int it = 0; it < 100; ++it) {
        double f = -T, fp = 0.0;
        for (int q = 0; q < H.nq; ++q) {
            const double e = H.a[q] * std::exp(H.b[q] * u);
            f += e;
            fp += H.b[q] * e;
        }
        if (!(fp > 0.0)) break;
        const double nu = u - f / fp;
        if (!(nu < u) || nu <= 0.0) break;
        if (u - nu <= 1e-16 * u) { u = nu; break; }
        u = nu;
    }
    return std::sqrt(u);
}

// Smallest float f >= 0 with F(f) >= T: for FP32 values, |r| >= f <=> F(|r|) >= T.
float series_threshold_up(const HostSeries &H, double T)
{
    if (std::isinf(T)) return INFINITY;
    if (T <= 1.0) return 0.0f;
    float f = (float)series_root(H, T);
    while (series_F(H, f) < T) f = std::nextafter(f, INFINITY);
    while (f > 0.0f && series_F(H, std::nextafter(f, 0.0f)) >= T) f = std::nextafter(f, 0.0f);
    return f;
}

// Largest float f >= 0 with F(f) <= T: for FP32 values, |r| <= f <=> F(|r|) <= T.
float series_threshold_down(const HostSeries &H, double T)
{
    if (std::isinf(T)) return INFINITY;
    if (T < 1.0) return -1.0f;                   // nothing satisfies F <= T < 1 (F >= 1)
    if (T == 1.0) return 0.0f;
    float f = (float)series_root(H, T);
    while (f > 0.0f && series_F(H, f) > T) f = std::nextafter(f, 0.0f);
    while (series_F(H, std::nextafter(f, INFINITY)) <= T) f = std::nextafter(f, INFINITY);
    return f;
}

float round_down_f(double w)
{
    if (std::isinf(w)) return INFINITY;
    float f = (float)w;
    if ((double)f > w) f = std::nextafter(f, -INFINITY);
    return f;
}

// Smallest float strictly above w.
float strictly_above_f(double w)
{
    float f = (float)w;
    if ((double)f < w) f = std::nextafter(f, INFINITY);
    if ((double)f == w) f = std::nextafter(f, INFINITY);
    return f;
}

// G(u) = sum_{q>=1} a_q exp((b_q - b_1) u): the q >= 1 terms without the
// common factor exp(b_1 u).
static double series_G(const HostSeries &H, double u)
{
    double acc = 0.0;
    for (int q = 1; q < H.nq; ++q) acc += H.a[q] * std::exp((H.b[q] - H.b[1]) * u);
    return acc;
}

// Chebyshev interpolant of G on [0, U] at degree deg (nodes of the first
// kind); returns its largest relative error on a grid of 129 points.
static double fit_G(const HostSeries &H, double U, int deg, double *coef)
{
    const int N = deg + 1;
    double fv[RL0_MAXPOLY];
    for (int j = 0; j < N; ++j) {
        const double tj = std::cos(M_PI * (j + 0.5) / N);
        fv[j] = series_G(H, 0.5 * (tj + 1.0) * U);
    }
    for (int k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc += fv[j] * std::cos(M_PI * k * (j + 0.5) / N);
        coef[k] = (k == 0 ? 1.0 : 2.0) * acc / N;
    }
    double worst = 0.0;
    for (int g = 0; g <= 128; ++g) {
        const double u = U * g / 128.0, t = 2.0 * u / U - 1.0;
        double b1 = 0.0, b2 = 0.0;
        for (int k = N - 1; k >= 1; --k) { const double b0 = 2.0 * t * b1 - b2 + coef[k]; b2 = b1; b1 = b0; }
        const double val = t * b1 - b2 + coef[0];
        const double ref = series_G(H, u);
        worst = std::fmax(worst, std::fabs(val - ref) / ref);
    }
    return worst;
}

// Device form of a series: FP32 coefficients, the 2^-40 cut, and the factored
// Chebyshev form of the q >= 1 terms when it reproduces them to 2e-9.
Series to_device_series(const HostSeries &H)
{
    Series S;
    std::memset(&S, 0, sizeof(S));
    S.nq = H.nq;
    for (int q = 0; q < H.nq; ++q) { S.a[q] = (float)H.a[q]; S.b[q] = (float)H.b[q]; }
    S.cut = series_threshold_up(H, std::ldexp(1.0, 40));   // p_breve < 2^-40 beyond
    const double U = (double)S.cut * (double)S.cut;
    if (H.nq >= 2 && std::isfinite(U) && U > 0.0) {
        double coef[RL0_MAXPOLY];
        for (int deg = 2; deg < RL0_MAXPOLY; ++deg) {
            if (fit_G(H, U, deg, coef) < 2e-9) {
                S.use_poly = 1;
                S.npoly = deg + 1;
                S.b1 = (float)H.b[1];
                S.inv_u2 = (float)(2.0 / U);
                for (int k = 0; k <= deg; ++k) S.poly[k] = (float)coef[k];
                break;
            }
        }
    }
    return S;
}

// Eqs. (finetune_c_quant), (finetune_c_cont).
double default_c(int quantised, double delta, double rho)
{
    if (quantised) {
        if (delta <= 0.05) return 0.01;
        if (rho <= 0.1) return 0.05;
        if (rho <= 0.2) return 0.075;
        return 0.1;
    }
    return delta <= 0.05 ? 0.01 : 0.025;
}

int resolve(int64_t n, int64_t m, int d, int64_t k, const rl0_params *in, Resolved *R)
{
    rl0_params p;
    std::memset(&p, 0, sizeof(p));
    if (in) p = *in;
    if (p.sigma_s == 0.0) p.sigma_s = 1.0;
    if (!(p.sigma_s > 0.0) || !(p.sigma_n >= 0.0) || !std::isfinite(p.sigma_n) || !std::isfinite(p.sigma_s))
        return RL0_ERR_INVALID_ARG;
    if (p.adaptive_k != 0 && p.adaptive_k != 1) return RL0_ERR_INVALID_ARG;
    if (p.adaptive_k && p.scorer != 0) return RL0_ERR_UNSUPPORTED;
    if (k < 1 || k > n) return RL0_ERR_INVALID_ARG;
    if (p.c == 0.0) p.c = default_c(p.quantised, (double)m / (double)n, (double)k / (double)m);
    if (!(p.c > 0.0 && p.c <= 1.0)) return RL0_ERR_INVALID_ARG;
    // reading: "more than d/2 rows agree" -- floor(d/2)+1 for the integer counts
    // of the quantised scores, d/2 for the soft counts of the continuous ones
    if (p.alpha == 0.0) p.alpha = p.quantised ? (double)(d / 2 + 1) : 0.5 * d;
    if (!(p.alpha > 0.0)) return RL0_ERR_INVALID_ARG;
    if (p.ell == 0) p.ell = 4;
    if (p.ell < 1 || p.ell > RL0_MAXQ - 2) return RL0_ERR_INVALID_ARG;
    if (p.noiseless_tol == 0.0) p.noiseless_tol = 1e-5;
    if (!(p.noiseless_tol > 0.0)) return RL0_ERR_INVALID_ARG;
    if (p.scorer != 0 && p.scorer != 1) return RL0_ERR_INVALID_ARG;
    if (p.scorer == 1 && (!p.mlp || !(p.sigma_n > 0.0) || d > 16)) return RL0_ERR_INVALID_ARG;
    if (p.scorer == 1 && !(p.mlp_threshold >= 0.0 && p.mlp_threshold < 1.0)) return RL0_ERR_INVALID_ARG;
    if (p.profile != 0 && p.profile != 1) return RL0_ERR_INVALID_ARG;
    if (p.anchor_rule != 0 && p.anchor_rule != 1) return RL0_ERR_INVALID_ARG;
    if (p.anchor_rule == 1 && p.scorer == 1) return RL0_ERR_UNSUPPORTED;
    // reading: t_r = 1 - r c for every r >= 0 with t_r > 0 (counted with a
    // tolerance so that c = 0.025 gives exactly 40 rounds)
    int nr = (int)std::ceil(1.0 / p.c - 1e-9);
    if (p.max_rounds > 0 && p.max_rounds < nr) nr = p.max_rounds;
    if (nr > RL0_MAX_ROUNDS) return RL0_ERR_UNSUPPORTED;
    R->p = p;
    R->nrounds = nr;
    R->indicator = p.quantised || p.sigma_n == 0.0;
    // Section "Stopping conditions": ||r||_1 <= E||eta||_1 = m sigma sqrt(2/pi);
    // reading: noiseless decodes stop at ||r||_1 <= tol ||y||_1
    R->stop_level = (p.sigma_n > 0.0) ? (double)m * p.sigma_n * std::sqrt(2.0 / M_PI) : 0.0;
    R->stop_rel = (p.sigma_n > 0.0) ? 0.0 : p.noiseless_tol;
    // learned decodes: a residual consistent with the noise, E||eta||_1 + 3 sqrt(Var||eta||_1)
    R->keep_level = R->stop_level + 3.0 * std::sqrt((double)m * p.sigma_n * p.sigma_n * (1.0 - 2.0 / M_PI));
    return RL0_OK;
}

// The decode context (minus the data pointers) and the per-round thresholds.
void fill_tables(int64_t m, int d, int64_t k, const Resolved &R, DecodeCtx *ctx, RoundThr *thr, int nthr,
                 double k_prior)
{
    const rl0_params &p = R.p;
    // the posteriors' sparsity: k, or the adaptive_k prior k0 (Alg. 2)
    const double rho = (k_prior > 0.0 ? k_prior : (double)k) / (double)m;
    const double s2 = p.sigma_s * p.sigma_s, n2 = p.sigma_n * p.sigma_n;
    std::memset(ctx, 0, sizeof(*ctx));
    ctx->k = k;
    ctx->alpha = (float)p.alpha;
    ctx->nrounds = R.nrounds;
    ctx->quantised = p.quantised;
    ctx->indicator = R.indicator;
    ctx->stop_level = R.stop_level;
    ctx->stop_rel = R.stop_rel;
    ctx->scorer = p.scorer;
    ctx->anchor_rule = p.anchor_rule;
    ctx->mlp = p.mlp;
    const double th = (p.mlp_threshold == 0.0) ? 0.5 : p.mlp_threshold;
    ctx->mlp_threshold = (float)th;
    ctx->logit_thr = (float)std::log(th / (1.0 - th));
    ctx->learned_need = 1.5f;
    ctx->inv_sn = (p.sigma_n > 0.0) ? (float)(1.0 / p.sigma_n) : 0.0f;
    // reading: at t = 1 the anchor test 1 - p_z(r) >= 1 needs p_z(r) = 0, which
    // never holds for sigma_n > 0, so the first round updates nothing
    ctx->skip_t1 = (p.sigma_n > 0.0) ? 1 : 0;
    ctx->drho = (float)(d * rho);
    HostSeries hz, he;
    if (p.sigma_n > 0.0) {
        hz = make_series(d * rho, s2, n2, p.ell);
        he = make_series(2.0 * d * rho, s2, 2.0 * n2, p.ell);
        ctx->pz = to_device_series(hz);
        ctx->pe = to_device_series(he);
        // every q >= 1 term has b_q >= b_1 and e^x >= 1 + x + x^2/2, so
        // p_e(D) = 1/F_e(D) <= 1 / (1 + (1 - a_0)(u + u^2/2)), u = b_1 D^2
        double bmin = INFINITY;
        for (int q = 1; q < he.nq; ++q) bmin = std::fmin(bmin, he.b[q]);
        ctx->pe_b1 = (float)bmin;
        ctx->pe_c1 = (float)(1.0 - he.a[0]);
    }
    for (int r = 0; r < nthr; ++r) {
        const double t = 1.0 - r * p.c;
        RoundThr T;
        T.t = (float)t;
        if (p.sigma_n == 0.0) {
            // p_breve is the indicator of |w| <= tol
            const float tol_dn = round_down_f(p.noiseless_tol);
            T.ta = strictly_above_f(p.noiseless_tol);       // p_z = 0  <=> |r| > tol
            T.te = tol_dn;                                  // p_e >= t <=> |D| <= tol (t in (0, 1])
            T.tz = (p.quantised && t >= 1.0) ? INFINITY : tol_dn;   // p_z >= 1 - t
        } else {
            // anchor: p_z(r) <= 1 - t <=> F_z(r) >= 1/(1-t);  q_z: p_z(r) >= 1 - t <=> F_z(r) <= 1/(1-t)
            const double Tz = (t >= 1.0) ? INFINITY : 1.0 / (1.0 - t);
            T.ta = series_threshold_up(hz, Tz);
            T.tz = series_threshold_down(hz, Tz);
            // q_e (quantised): p_e(D) >= t <=> F_e(D) <= 1/t
            T.te = series_threshold_down(he, 1.0 / t);
        }
        thr[r] = T;
    }
}

// Value of a non-negative FP16 bit pattern (0 .. 0x7c00; 0x7c00 is +inf).
static double half_bits_value(unsigned h)
{
    const unsigned e = h >> 10, f = h & 0x3ffu;
    if (e == 31) return INFINITY;
    if (e == 0) return std::ldexp((double)f, -24);
    return std::ldexp((double)(1024u + f), (int)e - 25);
}

// Lower bounds of p_z over the 16-bit residual codes.  A code of magnitude
// bits b stands for |r| < the FP16 value of b + 1, and p_breve_z is
// decreasing in |r| (1/p_breve_z = sum of positive a_q exp(b_q w^2)), so over
// bin c = b >> RL0_PZ_SHIFT the posterior is at least p_breve_z at the
// FP16 value of (c + 1) << RL0_PZ_SHIFT.  The factor 1 - 1e-5 covers the FP32
// evaluation on the device; past the series cut the device takes 0.
void pz_lower_bounds(int64_t m, int d, int64_t k, const Resolved &R, float *out, double k_prior)
{
    const rl0_params &p = R.p;
    if (!(p.sigma_n > 0.0)) {
        for (int c = 0; c < RL0_PZ_BINS; ++c) out[c] = 0.0f;
        return;
    }
    const double rho = (k_prior > 0.0 ? k_prior : (double)k) / (double)m;
    const HostSeries hz = make_series(d * rho, p.sigma_s * p.sigma_s, p.sigma_n * p.sigma_n, p.ell);
    const double cut = (double)to_device_series(hz).cut;
    for (int c = 0; c < RL0_PZ_BINS; ++c) {
        const double U = half_bits_value((unsigned)(c + 1) << RL0_PZ_SHIFT);
        out[c] = (U > cut) ? 0.0f : (float)((1.0 - 1e-5) / series_F(hz, U));
    }
}

// Alg. 2's adaptive_k step from the support of x_hat (index, value pairs in
// ascending index): k0 = k - sum_j (1 - p_z(x_hat_j)) in FP64, floored at
// m/100, with p_z the posterior at the prior k_prior (reading: the printed
// k - sum_j p_z(x_hat_j) would count almost every zero entry).
double adaptive_k0(int64_t m, int d, int64_t k, const Resolved &R, double k_prior, const float *vals, int64_t count)
{
    const rl0_params &p = R.p;
    double s = 0.0;
    if (p.sigma_n > 0.0) {
        const double rho = k_prior / (double)m;
        const HostSeries hz = make_series(d * rho, p.sigma_s * p.sigma_s, p.sigma_n * p.sigma_n, p.ell);
        for (int64_t e = 0; e < count; ++e)
            if (vals[e] != 0.0f) s += 1.0 - 1.0 / series_F(hz, (double)vals[e]);
    } else {
        // noiseless: p_z is the indicator of |w| <= tol
        for (int64_t e = 0; e < count; ++e)
            if (std::fabs((double)vals[e]) > p.noiseless_tol) s += 1.0;
    }
    const double k0 = (double)k - s;
    const double lo = std::floor((double)m / 100.0);
    return k0 > lo ? k0 : lo;
}

}  // namespace rl0

/*
 * cse_oracle.c -- plain, slow, FP64 CPU oracle for the Continuous Simulation
 * Extension (CSE) hot path of Yang, Thompson & Sklar, "Guarantees for
 * Comprehensive Simulation Assessment of Statistical Methods" (arXiv 2212.10042).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path in paper_2212_10042_gb300/csrc.
 *
 * What it computes, in the paper's order:
 *   - Philox4x32-10 counter-based uniforms (Salmon et al., SC'11), used as common
 *     random numbers shared by every grid point (Sec. 7.3 "Calibration on a
 *     General Bounded Space", CRN remark; Fig. calibration-z-test caption).
 *   - Bernoulli draws of the embedded i.i.d. model (Sec. 9, adaptive embedding of
 *     binomial arms): patient j of arm a succeeds iff u < floor(2^32 sigmoid(theta_a)).
 *     Success counts by a LINEAR SCAN over the patients (not a binary search).
 *   - Test statistics S(X), rejection iff S < lambda (Sec. 7, f_lambda = P(S<lambda)).
 *   - Reject count R, score sums sum 1{rej} (T - grad A(theta)) (Ex. exp-fam:
 *     g_theta(x) = T(x)'theta, so grad log p = T - grad A).
 *   - Clopper-Pearson upper bound (Eq. clopper-pearson:def), here by an explicit
 *     binomial-CDF sum in log space, inverted by bisection + Newton.
 *   - Tilewise optimised Tilt-Bound (Thm. tilt-bound, Eq. tilt-bound:exp-fam,
 *     Eq. optimized-tilt-bound-tile), sup over the 2^d box vertices (Thm. 3),
 *     inf over q by golden-section search in s = log q (Thm. 2 quasi-convexity)
 *     followed by Newton steps on the analytic derivative.
 *   - Calibration target alpha' (Eq. tilt-bound-inv, Eq. tile-calibration-final),
 *     order statistic S_(floor((N+1)alpha')) (Eq. calibrated-threshold) by a full
 *     sort, and the minimum over tiles (Eq. calibrated-threshold-final).
 *   - The Bayesian four-arm selection design's posterior in FP64 (Sec. 10.1
 *     hierarchical model; each arm's likelihood by the normal approximation of
 *     its empirical logit, s2 on 16 log-spaced quadrature nodes).
 *
 * Floating point: FP64 everywhere except the two z statistics, whose definition
 * here is an FP32 expression evaluated with correctly rounded single
 * precision operations in a fixed order (compile with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by two constants,
 * XORs the high halves into words 1 and 3 together with the round key, and
 * permutes; the key is bumped by the Weyl constants between rounds.          */
/* ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform word for sim k, arm a, patient j: counter (k, a, j/4, 0), key = seed. */
uint32_t orc_uniform(uint64_t seed, uint32_t k, uint32_t a, uint32_t j)
{
    uint32_t ctr[4] = { k, a, j / 4u, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[j % 4u];
}

/* Tie-break word of sim k for the randomised test (Sec. 7: an independent
 * uniform adjoined to the sample space): word 0 of Philox4x32-10(counter
 * (k, 0, 0, 1), key = seed).  The patients' draws use counter word 3 = 0, so no
 * counter is shared. */
uint32_t orc_tiebreak(uint64_t seed, uint32_t k)
{
    uint32_t ctr[4] = { k, 0u, 0u, 1u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* Success threshold t(theta) = floor(2^32 sigmoid(theta)), clamped to [0, 2^32-1];
 * a draw u succeeds iff u < t, so P(success) = t / 2^32. */
uint32_t orc_threshold(double theta)
{
    double p = 1.0 / (1.0 + exp(-theta));
    double y = p * 4294967296.0;
    if (!(y >= 0.0)) return 0u;
    if (y >= 4294967295.0) return 4294967295u;
    return (uint32_t)floor(y);
}

/* ------------------------------------------------------------------------- */
/* Design description (the oracle's own struct).                               */
/* ------------------------------------------------------------------------- */
enum { ORC_STAT_ONE_ARM_Z = 0, ORC_STAT_TWO_ARM_POOLED_Z = 1, ORC_STAT_BAYES4 = 2, ORC_STAT_BERRY4 = 3 };

typedef struct {
    int32_t stat;       /* one of ORC_STAT_* */
    int32_t d;          /* number of arms (1, 2 or 4) */
    int32_t n_looks;    /* 1..3 */
    int32_t look_n[3];  /* cumulative patients per arm at each look */
    double p0;          /* one-arm z-test null proportion */
    double drop;        /* Bayes design: interim drop threshold */
    uint64_t seed;
    double tnull[4];    /* basket design: logit of each arm's null response rate */
} orc_design;

/* ------------------------------------------------------------------------- */
/* Test statistics.  Small S rejects (Sec. 7: reject iff S(X) < lambda).        */
/* ------------------------------------------------------------------------- */

/* One-arm z-test, S = -(x - n p0) / sqrt(n p0 (1 - p0)), evaluated in FP32. */
double orc_stat_one_arm(int32_t x, int32_t n, double p0)
{
    float fp0 = (float)p0;
    float fn = (float)n;
    float num = (float)x - fn * fp0;
    float var = fn * fp0;
    var = var * (1.0f - fp0);
    float z = num / sqrtf(var);
    return (double)(-z);
}

/* Two-arm pooled z-test of arm 1 (treatment) against arm 0 (control),
 * S = -z, z = (p1 - p0) / sqrt(pbar (1 - pbar) (1/n0 + 1/n1)), in FP32;
 * z = 0 when the pooled variance is zero (x0 + x1 in {0, n0 + n1}). */
double orc_stat_two_arm(int32_t x0, int32_t x1, int32_t n0, int32_t n1)
{
    float fn0 = (float)n0, fn1 = (float)n1;
    float p0 = (float)x0 / fn0;
    float p1 = (float)x1 / fn1;
    float pb = (float)(x0 + x1) / (fn0 + fn1);
    float inv = 1.0f / fn0 + 1.0f / fn1;
    float var = pb * (1.0f - pb);
    var = var * inv;
    float z = 0.0f;
    if (var > 0.0f) z = (p1 - p0) / sqrtf(var);
    return (double)(-z);
}

/* --- Bayesian hierarchical model, Sec. 10.1: theta_i ~ N(mu, s2),
 *     mu ~ N(-1.34, 100), s2 ~ InvGamma(0.0005, 0.000005); each arm's likelihood
 *     replaced by the normal approximation of its empirical logit; s2 integrated
 *     on 16 log-spaced nodes in [1e-6, 1e3] (trapezoid in log s2). --- */
#define ORC_MU0 (-1.34)
#define ORC_TAU2 100.0
#define ORC_IG_A 0.0005
#define ORC_IG_B 0.000005
#define ORC_NODES 16

static double orc_norm_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* P(theta_i > theta_0 | data), i = 1..3, written to P[0..2]. */
void orc_bayes4_posterior(const int32_t x[4], const int32_t n[4], double P[3])
{
    double th[4], s2[4];
    for (int i = 0; i < 4; ++i) {
        double xs = (double)x[i] + 0.5, fs = (double)(n[i] - x[i]) + 0.5;
        th[i] = log(xs / fs);
        s2[i] = 1.0 / xs + 1.0 / fs;
    }
    double lo = log(1e-6), hi = log(1e3);
    double logw[ORC_NODES], pij[ORC_NODES][3];
    for (int j = 0; j < ORC_NODES; ++j) {
        double L = lo + (hi - lo) * (double)j / (double)(ORC_NODES - 1);
        double sig2 = exp(L);
        double W = 0.0, Sr = 0.0, Srr = 0.0, Sth = 0.0, logdet = 0.0;
        for (int i = 0; i < 4; ++i) {
            double wi = 1.0 / (sig2 + s2[i]);
            double r = th[i] - ORC_MU0;
            W += wi;
            Sr += wi * r;
            Srr += wi * r * r;
            Sth += wi * th[i];
            logdet += log(sig2 + s2[i]);
        }
        double prec = 1.0 / ORC_TAU2 + W;
        double quad = Srr - Sr * Sr / prec;
        logdet += log(1.0 + ORC_TAU2 * W);
        double trap = (j == 0 || j == ORC_NODES - 1) ? log(0.5) : 0.0;
        /* prior density of s2 times the Jacobian d s2 = s2 d log s2 */
        double logprior = -(ORC_IG_A + 1.0) * L - ORC_IG_B / sig2 + L;
        logw[j] = trap + logprior - 0.5 * logdet - 0.5 * quad;
        double mmu = (ORC_MU0 / ORC_TAU2 + Sth) / prec;
        double vmu = 1.0 / prec;
        double c[4], v[4], e[4];
        for (int i = 0; i < 4; ++i) {
            c[i] = s2[i] / (s2[i] + sig2);
            v[i] = s2[i] * sig2 / (s2[i] + sig2);
            e[i] = (1.0 - c[i]) * th[i] + c[i] * mmu;
        }
        for (int i = 1; i < 4; ++i) {
            double md = e[i] - e[0];
            double dc = c[i] - c[0];
            double vd = v[i] + v[0] + dc * dc * vmu;
            pij[j][i - 1] = orc_norm_cdf(md / sqrt(vd));
        }
    }
    double mx = logw[0];
    for (int j = 1; j < ORC_NODES; ++j) if (logw[j] > mx) mx = logw[j];
    double tot = 0.0, acc[3] = { 0.0, 0.0, 0.0 };
    for (int j = 0; j < ORC_NODES; ++j) {
        double w = exp(logw[j] - mx);
        tot += w;
        for (int i = 0; i < 3; ++i) acc[i] += w * pij[j][i];
    }
    for (int i = 0; i < 3; ++i) P[i] = acc[i] / tot;
}

/* Four-arm selection design on cumulative counts xl[look][arm]:
 * interim looks drop treatment i when P_i < drop (data frozen, still in the
 * model); all treatments dropped stops without rejection; at the final look
 * S = min over active i with hypothesis H_i in null_mask of (1 - P_i).
 * Returns +INFINITY when no true-null arm can be rejected. */
/* Basket design (Sec. 10.1, Bayesian basket trial): four arms of n patients, one
 * analysis; the offset log-odds theta_i = logit(p_i) - t_i share the hierarchy of
 * the four-arm design (theta_i ~ N(mu, s2), mu ~ N(-1.34, 100), s2 ~ IG(0.0005,
 * 0.000005)), each arm's likelihood by the normal approximation of its empirical
 * logit minus t_i; mu integrated exactly, s2 on the same nodes.
 * P[i] = P(theta_i > 0 | x) = P(p_i > p_0i | x) for all four arms. */
void orc_berry_posterior(const int32_t x[4], int32_t n, const double tnull[4], double P[4])
{
    double th[4], s2[4];
    for (int i = 0; i < 4; ++i) {
        double xs = (double)x[i] + 0.5, fs = (double)(n - x[i]) + 0.5;
        th[i] = log(xs / fs) - tnull[i];
        s2[i] = 1.0 / xs + 1.0 / fs;
    }
    double lo = log(1e-6), hi = log(1e3);
    double logw[ORC_NODES], pj[ORC_NODES][4];
    for (int j = 0; j < ORC_NODES; ++j) {
        double L = lo + (hi - lo) * (double)j / (double)(ORC_NODES - 1);
        double sig2 = exp(L);
        double W = 0.0, Sr = 0.0, Srr = 0.0, Sth = 0.0, logdet = 0.0;
        for (int i = 0; i < 4; ++i) {
            double wi = 1.0 / (sig2 + s2[i]);
            double r = th[i] - ORC_MU0;
            W += wi;
            Sr += wi * r;
            Srr += wi * r * r;
            Sth += wi * th[i];
            logdet += log(sig2 + s2[i]);
        }
        double prec = 1.0 / ORC_TAU2 + W;
        double quad = Srr - Sr * Sr / prec;
        logdet += log(1.0 + ORC_TAU2 * W);
        double trap = (j == 0 || j == ORC_NODES - 1) ? log(0.5) : 0.0;
        double logprior = -(ORC_IG_A + 1.0) * L - ORC_IG_B / sig2 + L;
        logw[j] = trap + logprior - 0.5 * logdet - 0.5 * quad;
        double mmu = (ORC_MU0 / ORC_TAU2 + Sth) / prec;
        double vmu = 1.0 / prec;
        for (int i = 0; i < 4; ++i) {
            /* theta_i | mu, s2, x ~ N((1-c) th_i + c mu, s2_i s2 / (s2_i + s2)), c = s2_i / (s2_i + s2);
             * over mu ~ N(mmu, vmu): mean (1-c) th_i + c mmu, variance v + c^2 vmu */
            double c = s2[i] / (s2[i] + sig2);
            double v = s2[i] * sig2 / (s2[i] + sig2) + c * c * vmu;
            double m = (1.0 - c) * th[i] + c * mmu;
            pj[j][i] = orc_norm_cdf(m / sqrt(v));
        }
    }
    double mx = logw[0];
    for (int j = 1; j < ORC_NODES; ++j) if (logw[j] > mx) mx = logw[j];
    double tot = 0.0, acc[4] = { 0.0, 0.0, 0.0, 0.0 };
    for (int j = 0; j < ORC_NODES; ++j) {
        double w = exp(logw[j] - mx);
        tot += w;
        for (int i = 0; i < 4; ++i) acc[i] += w * pj[j][i];
    }
    for (int i = 0; i < 4; ++i) P[i] = acc[i] / tot;
}

/* Basket statistic: S = min over the arms of the tile's null set of
 * (1 - P(theta_i > 0 | x)); reject iff S < lambda (lambda = 0.15 for the 85%
 * rule); +inf when the set is empty. */
double orc_berry_stat(const orc_design* D, const int32_t x[4], uint32_t null_mask)
{
    double P[4];
    orc_berry_posterior(x, D->look_n[D->n_looks - 1], D->tnull, P);
    double S = INFINITY;
    for (int i = 0; i < 4; ++i)
        if ((null_mask >> i) & 1u) S = fmin(S, 1.0 - P[i]);
    return S;
}

double orc_bayes4_stat(const orc_design* D, const int32_t xl[3][4], uint32_t null_mask)
{
    int active[4] = { 1, 1, 1, 1 };
    int32_t fx[4], fn[4];
    for (int l = 0; l < D->n_looks; ++l) {
        int32_t x[4], n[4];
        for (int i = 0; i < 4; ++i) {
            if (i == 0 || active[i]) {
                x[i] = xl[l][i];
                n[i] = D->look_n[l];
            } else {
                x[i] = fx[i];
                n[i] = fn[i];
            }
        }
        double P[3];
        orc_bayes4_posterior(x, n, P);
        if (l < D->n_looks - 1) {
            int any = 0;
            for (int i = 1; i < 4; ++i) {
                if (active[i] && P[i - 1] < D->drop) {
                    active[i] = 0;
                    fx[i] = x[i];
                    fn[i] = n[i];
                }
                any |= active[i];
            }
            if (!any) return INFINITY;
        } else {
            double S = INFINITY;
            for (int i = 1; i < 4; ++i) {
                if (active[i] && ((null_mask >> (i - 1)) & 1u)) {
                    double s = 1.0 - P[i - 1];
                    if (s < S) S = s;
                }
            }
            return S;
        }
    }
    return INFINITY;
}

/* ------------------------------------------------------------------------- */
/* Simulation (Sec. 6.1 / 7.1): per tile, per sim: counts -> S -> S < lambda.   */
/* ------------------------------------------------------------------------- */

static int orc_n_max(const orc_design* D) { return D->look_n[D->n_looks - 1]; }

/* Cumulative success counts of one sim: x[l*4 + a] = #{j < look_n[l] : u < t_a}. */
void orc_counts(const orc_design* D, const uint32_t* t, uint32_t k, int32_t* x)
{
    for (int a = 0; a < D->d; ++a) {
        int32_t c = 0;
        int j = 0;
        for (int l = 0; l < D->n_looks; ++l) {
            for (; j < D->look_n[l]; ++j)
                if (orc_uniform(D->seed, k, (uint32_t)a, (uint32_t)j) < t[a]) c += 1;
            x[l * 4 + a] = c;
        }
    }
}

static double orc_statistic(const orc_design* D, const int32_t* x, uint32_t null_mask)
{
    int last = D->n_looks - 1;
    int nm = orc_n_max(D);
    switch (D->stat) {
    case ORC_STAT_ONE_ARM_Z:
        return orc_stat_one_arm(x[last * 4 + 0], nm, D->p0);
    case ORC_STAT_TWO_ARM_POOLED_Z:
        return orc_stat_two_arm(x[last * 4 + 0], x[last * 4 + 1], nm, nm);
    case ORC_STAT_BERRY4:
        return orc_berry_stat(D, x + last * 4, null_mask);
    case ORC_STAT_BAYES4: {
        int32_t xl[3][4];
        for (int l = 0; l < 3; ++l)
            for (int a = 0; a < 4; ++a) xl[l][a] = (l < D->n_looks) ? x[l * 4 + a] : 0;
        return orc_bayes4_stat(D, (const int32_t(*)[4])xl, null_mask);
    }
    }
    return NAN;
}

static double orc_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/*
 * Simulate every tile: R[i] = sum_k 1{S_ik < lambda}, Xrej[i][a] =
 * sum_k 1{rej} T_a (T_a = successes of arm a over all n_max patients),
 * score[i][a] = Xrej - n_max sigmoid(theta_a) R  (the score-function sum
 * sum_k 1{rej}(T - grad A(theta))).  If S_out is non-NULL, S_ik is stored at
 * S_out[S_off[i] + k].  theta is [n_tiles][d].
 */
int orc_simulate(const orc_design* D, int64_t n_tiles, const double* theta,
                 const uint32_t* null_mask, const int32_t* K, double lambda,
                 int64_t* R, int64_t* Xrej, double* score,
                 double* S_out, const int64_t* S_off)
{
    int d = D->d;
    int nm = orc_n_max(D);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < n_tiles; ++i) {
        uint32_t t[4] = { 0, 0, 0, 0 };
        for (int a = 0; a < d; ++a) t[a] = orc_threshold(theta[i * d + a]);
        int64_t r = 0, xr[4] = { 0, 0, 0, 0 };
        for (int32_t k = 0; k < K[i]; ++k) {
            int32_t x[12];
            orc_counts(D, t, (uint32_t)k, x);
            double S = orc_statistic(D, x, null_mask[i]);
            if (S_out) S_out[S_off[i] + k] = S;
            if (S < lambda) {
                r += 1;
                for (int a = 0; a < d; ++a) xr[a] += x[(D->n_looks - 1) * 4 + a];
            }
        }
        if (R) R[i] = r;
        for (int a = 0; a < d; ++a) {
            if (Xrej) Xrej[i * d + a] = xr[a];
            if (score) score[i * d + a] = (double)xr[a] - (double)nm * orc_sigmoid(theta[i * d + a]) * (double)r;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Clopper-Pearson upper bound (Eq. clopper-pearson:def):                     */
/*   u = Beta^{-1}(1 - delta; R + 1, N - R), i.e. the u with                  */
/*   P(Binom(N, u) <= R) = delta.  R = N gives 1.                             */
/* ------------------------------------------------------------------------- */

/* log P(Binom(N, u) <= R) by summing the pmf, log C(N,j) accumulated with a
 * compensated sum, then log-sum-exp. */
static double orc_log_binom_cdf(int64_t R, int64_t N, double u)
{
    if (u <= 0.0) return 0.0;
    if (u >= 1.0) return (R >= N) ? 0.0 : -INFINITY;
    double lq = log1p(-u), lu = log(u);
    double logit = lu - lq;
    double base = (double)N * lq;
    /* first pass: max term */
    double lc = 0.0, comp = 0.0, mx = -INFINITY;
    double* terms = (double*)malloc(sizeof(double) * (size_t)(R + 1));
    for (int64_t j = 0; j <= R; ++j) {
        double lp = base + lc + (double)j * logit;
        terms[j] = lp;
        if (lp > mx) mx = lp;
        /* lc += log((N - j) / (j + 1)), Kahan-compensated */
        double inc = log((double)(N - j)) - log((double)(j + 1));
        double y = inc - comp;
        double tt = lc + y;
        comp = (tt - lc) - y;
        lc = tt;
    }
    double s = 0.0;
    for (int64_t j = 0; j <= R; ++j) s += exp(terms[j] - mx);
    free(terms);
    return mx + log(s);
}

double orc_cp_upper(int64_t R, int64_t N, double delta)
{
    if (R >= N) return 1.0;
    double ld = log(delta);
    double lo = 0.0, hi = 1.0;
    /* F(u) = P(Binom(N,u) <= R) is decreasing in u.  Bisection on log F. */
    double u = ((double)R + 1.0) / ((double)N + 1.0);
    for (int it = 0; it < 200; ++it) {
        double f = orc_log_binom_cdf(R, N, u) - ld;
        if (f > 0.0) lo = u; else hi = u;
        if (hi - lo <= 1e-17 * hi) break;
        /* Newton step in log space: d/du log F = -pdf(u) / F(u),
         * pdf = Beta(R+1, N-R) density = (N-R) C(N,R) u^R (1-u)^(N-R-1). */
        double lpdf = log((double)(N - R)) + lgamma((double)N + 1.0) - lgamma((double)R + 1.0)
                      - lgamma((double)(N - R) + 1.0) + (double)R * log(u) + (double)(N - R - 1) * log1p(-u);
        double dlogF = -exp(lpdf - (f + ld));
        double un = u - f / dlogF;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        if (fabs(un - u) <= 1e-17 * u) { u = un; break; }
        u = un;
    }
    return u;
}

/* Lower Clopper-Pearson bound: l = Beta^{-1}(delta; R, N - R + 1), i.e. the l
 * with P(Binom(N, l) >= R) = delta; R = 0 gives 0.  Written from the upper
 * tail (its own sum over j = R..N), not from the CDF above. */
/* log C(N, R) as a compensated sum of min(R, N-R) log ratios (a difference
 * of two lgamma values of size N log N would lose ~N log N * 1e-16). */
static double orc_log_choose(int64_t N, int64_t R)
{
    int64_t m = (R < N - R) ? R : N - R;
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double inc = log((double)(N - i)) - log((double)(i + 1));
        double y = inc - comp;
        double t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    return s;
}

static double orc_log_binom_sf(int64_t R, int64_t N, double u)
{
    if (R <= 0) return 0.0;
    if (u <= 0.0) return -INFINITY;
    if (u >= 1.0) return 0.0;
    double lq = log1p(-u), lu = log(u);
    double logit = lu - lq;
    /* log pmf(R), then log pmf(j+1) = log pmf(j) + log((N-j)/(j+1)) + logit,
     * the increments Kahan-compensated.  Past the mode the terms fall
     * geometrically (ratio < 1), so once a term is 60 below the largest the
     * rest of the tail is below e^-60 of the sum and the loop stops. */
    double lp = orc_log_choose(N, R) + (double)R * lu + (double)(N - R) * lq;
    double mode = ((double)N + 1.0) * u;
    int64_t cap = N - R + 1;
    double* terms = (double*)malloc(sizeof(double) * (size_t)cap);
    double mx = -INFINITY, comp = 0.0;
    int64_t n = 0;
    for (int64_t j = R; j <= N; ++j) {
        terms[n++] = lp;
        if (lp > mx) mx = lp;
        if ((double)j > mode && lp < mx - 60.0) break;
        if (j == N) break;
        double inc = log((double)(N - j)) - log((double)(j + 1)) + logit;
        double y = inc - comp;
        double tt = lp + y;
        comp = (tt - lp) - y;
        lp = tt;
    }
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += exp(terms[j] - mx);
    free(terms);
    return mx + log(s);
}

double orc_cp_lower(int64_t R, int64_t N, double delta)
{
    if (R <= 0) return 0.0;
    double ld = log(delta);
    double lo = 0.0, hi = 1.0;
    /* S(u) = P(Binom(N,u) >= R) is increasing in u.  Bisection on log S,
     * with Newton steps: d/du log S = pdf(u) / S(u), pdf the Beta(R, N-R+1)
     * density N C(N-1, R-1) u^(R-1) (1-u)^(N-R). */
    double u = (double)R / ((double)N + 1.0);
    for (int it = 0; it < 200; ++it) {
        double f = orc_log_binom_sf(R, N, u) - ld;
        if (f < 0.0) lo = u; else hi = u;
        if (hi - lo <= 1e-17 * hi) break;
        double lpdf = log((double)N) + lgamma((double)N) - lgamma((double)R) - lgamma((double)(N - R) + 1.0)
                      + (double)(R - 1) * log(u) + (double)(N - R) * log1p(-u);
        double dlogS = exp(lpdf - (f + ld));
        double un = u - f / dlogS;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        if (fabs(un - u) <= 1e-17 * u) { u = un; break; }
        u = un;
    }
    return u;
}

/* ------------------------------------------------------------------------- */
/* Tilt-Bound (Thm. tilt-bound; Eq. tilt-bound:exp-fam):                       */
/*   log U(theta0, v, q, a) = (1 - 1/q) log a + psi(q)/q - psi(1),            */
/*   psi(q) = A(theta0 + q v) - A(theta0).                                    */
/* Families: 0 = binomial arms on the logit scale, A = sum_a n_a softplus;    */
/*           1 = normal location, A = sum_a n_a theta_a^2 / 2 (test family). */
/* ------------------------------------------------------------------------- */

static double orc_softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

typedef struct {
    int family;
    int d;
    double n[4];
    double th0[4];
} orc_fam;

static double orc_A(const orc_fam* F, const double* th)
{
    double s = 0.0;
    for (int a = 0; a < F->d; ++a) {
        if (F->family == 0) s += F->n[a] * orc_softplus(th[a]);
        else s += F->n[a] * 0.5 * th[a] * th[a];
    }
    return s;
}

/* psi(q) = A(theta0 + q v) - A(theta0), summed per arm. */
static double orc_psi(const orc_fam* F, const double* v, double q)
{
    double s = 0.0;
    for (int a = 0; a < F->d; ++a) {
        double x = F->th0[a] + q * v[a];
        if (F->family == 0) s += F->n[a] * (orc_softplus(x) - orc_softplus(F->th0[a]));
        else s += F->n[a] * 0.5 * (x * x - F->th0[a] * F->th0[a]);
    }
    return s;
}

/* d psi / d q = v . grad A(theta0 + q v) */
static double orc_dpsi(const orc_fam* F, const double* v, double q)
{
    double s = 0.0;
    for (int a = 0; a < F->d; ++a) {
        double x = F->th0[a] + q * v[a];
        if (F->family == 0) s += F->n[a] * orc_sigmoid(x) * v[a];
        else s += F->n[a] * x * v[a];
    }
    return s;
}

/* d^2 psi / d q^2 = v' Hess A(theta0 + q v) v */
static double orc_d2psi(const orc_fam* F, const double* v, double q)
{
    double s = 0.0;
    for (int a = 0; a < F->d; ++a) {
        double x = F->th0[a] + q * v[a];
        if (F->family == 0) {
            double p = orc_sigmoid(x);
            s += F->n[a] * p * (1.0 - p) * v[a] * v[a];
        } else s += F->n[a] * v[a] * v[a];
    }
    return s;
}

/* lim_{q -> inf} psi(q) / q: binomial sum_a n_a max(v_a, 0); normal +inf unless v = 0. */
static double orc_psi_slope_inf(const orc_fam* F, const double* v)
{
    double s = 0.0;
    for (int a = 0; a < F->d; ++a) {
        if (F->family == 0) s += F->n[a] * fmax(v[a], 0.0);
        else if (v[a] != 0.0) return INFINITY;
    }
    return s;
}

static void orc_vertex(const double* h, int d, int m, double* v)
{
    for (int a = 0; a < d; ++a) v[a] = ((m >> a) & 1) ? h[a] : -h[a];
}

#define ORC_SMAX 40.0

/* g(q) = max over vertices of log U; *arg = maximising vertex */
static double orc_tilt_g(const orc_fam* F, const double* h, double loga, double q, int* arg)
{
    int nv = 1 << F->d;
    double best = -INFINITY;
    int bi = 0;
    for (int m = 0; m < nv; ++m) {
        double v[4];
        orc_vertex(h, F->d, m, v);
        double L = (1.0 - 1.0 / q) * loga + orc_psi(F, v, q) / q - orc_psi(F, v, 1.0);
        if (L > best) { best = L; bi = m; }
    }
    if (arg) *arg = bi;
    return best;
}

static double orc_tilt_g_inf(const orc_fam* F, const double* h, double loga)
{
    int nv = 1 << F->d;
    double best = -INFINITY;
    for (int m = 0; m < nv; ++m) {
        double v[4];
        orc_vertex(h, F->d, m, v);
        double L = loga + orc_psi_slope_inf(F, v) - orc_psi(F, v, 1.0);
        if (L > best) best = L;
    }
    return best;
}

/* Tilewise optimised Tilt-Bound in log form: log inf_q max_v U(theta0, v, q, a)
 * from log a (so that a = 1 - l with small l keeps its digits: log a = log1p(-l)). */
void orc_tilt_bound_log(int family, int d, const double* nvec, const double* theta0,
                        const double* h, double loga, double* logbound, double* qstar)
{
    orc_fam F;
    F.family = family; F.d = d;
    for (int i = 0; i < d; ++i) { F.n[i] = nvec[i]; F.th0[i] = theta0[i]; }
    if (loga >= 0.0) { *logbound = 0.0; *qstar = 1.0; return; }
    if (loga == -INFINITY) { *logbound = -INFINITY; *qstar = INFINITY; return; }
    /* golden-section search for the minimum of g(e^s) on [0, SMAX] */
    const double gr = 0.5 * (sqrt(5.0) - 1.0);
    double lo = 0.0, hi = ORC_SMAX;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double f1 = orc_tilt_g(&F, h, loga, exp(x1), NULL);
    double f2 = orc_tilt_g(&F, h, loga, exp(x2), NULL);
    while (hi - lo > 1e-15 * fmax(1.0, fabs(hi))) {
        if (f1 <= f2) {
            hi = x2; x2 = x1; f2 = f1;
            x1 = hi - gr * (hi - lo);
            f1 = orc_tilt_g(&F, h, loga, exp(x1), NULL);
        } else {
            lo = x1; x1 = x2; f1 = f2;
            x2 = lo + gr * (hi - lo);
            f2 = orc_tilt_g(&F, h, loga, exp(x2), NULL);
        }
    }
    double s = 0.5 * (lo + hi);
    double q = exp(s);
    int arg;
    double g = orc_tilt_g(&F, h, loga, q, &arg);
    /* minimiser beyond the search range: use the q -> inf limit (Thm. 2, a -> 0 case) */
    if (s > ORC_SMAX - 1e-6) {
        double ginf = orc_tilt_g_inf(&F, h, loga);
        if (ginf <= g) { *logbound = ginf; *qstar = INFINITY; return; }
    }
    /* Newton on the active vertex: dL/dq = [log a + q psi'(q) - psi(q)] / q^2 */
    double v[4];
    orc_vertex(h, d, arg, v);
    for (int it = 0; it < 3; ++it) {
        double N = loga + q * orc_dpsi(&F, v, q) - orc_psi(&F, v, q);
        double dN = q * orc_d2psi(&F, v, q);
        if (!(dN > 0.0)) break;
        double qn = q - N / dN;
        if (!(qn >= 1.0)) break;
        double gn = orc_tilt_g(&F, h, loga, qn, NULL);
        /* accept while the value does not rise beyond rounding (a kink would) */
        if (gn <= g + 8e-16 * fmax(1.0, fabs(g))) { q = qn; g = fmin(g, gn); } else break;
    }
    if (q < 1.0) q = 1.0;
    /* q = 1 gives U = 1 exactly, so the infimum is at most 1 (log 0) */
    if (g > 0.0) { g = 0.0; q = 1.0; }
    *logbound = g;
    *qstar = q;
}

/* Tilewise optimised Tilt-Bound: inf_q max_v U(theta0, v, q, a). */
void orc_tilt_bound(int family, int d, const double* nvec, const double* theta0,
                    const double* h, double a, double* bound, double* qstar)
{
    if (a >= 1.0) { *bound = 1.0; *qstar = 1.0; return; }
    if (a <= 0.0) { *bound = 0.0; *qstar = INFINITY; return; }
    double lb;
    orc_tilt_bound_log(family, d, nvec, theta0, h, log(a), &lb, qstar);
    *bound = exp(lb);
}

/* Lower Tilt-Bound (Rem. extension-lower): applying the Tilt-Bound to 1 - F
 * gives f(theta0 + v) >= 1 - (1 - f(theta0))^(1-1/q) exp[psi(q)/q - psi(1)];
 * the tilewise optimum over q of the minimum over the box is
 * 1 - inf_q max_v U(theta0, v, q, 1 - l) for a lower estimate l of f(theta0). */
void orc_tilt_lower(int family, int d, const double* nvec, const double* theta0,
                    const double* h, double l, double* lower, double* qstar)
{
    if (l <= 0.0) { *lower = 0.0; *qstar = 1.0; return; }
    if (l >= 1.0) { *lower = 1.0; *qstar = INFINITY; return; }
    double lb;
    orc_tilt_bound_log(family, d, nvec, theta0, h, log1p(-l), &lb, qstar);
    *lower = (lb >= 0.0) ? 0.0 : -expm1(lb);
}

/* Inverted Tilt-Bound (Eq. tilt-bound-inv), log form:
 *   log U^{-1}(q) = q/(q-1) [log alpha - psi(q)/q + psi(1)];
 * alpha' = sup_q min_v U^{-1} (Eq. tile-calibration-final). */
static double orc_inv_h(const orc_fam* F, const double* h, double logal, double q, int* arg)
{
    int nv = 1 << F->d;
    double best = INFINITY;
    int bi = 0;
    for (int m = 0; m < nv; ++m) {
        double v[4];
        orc_vertex(h, F->d, m, v);
        double M = q / (q - 1.0) * (logal - orc_psi(F, v, q) / q + orc_psi(F, v, 1.0));
        if (M < best) { best = M; bi = m; }
    }
    if (arg) *arg = bi;
    return best;
}

static double orc_inv_h_inf(const orc_fam* F, const double* h, double logal)
{
    int nv = 1 << F->d;
    double best = INFINITY;
    for (int m = 0; m < nv; ++m) {
        double v[4];
        orc_vertex(h, F->d, m, v);
        double M = logal - orc_psi_slope_inf(F, v) + orc_psi(F, v, 1.0);
        if (M < best) best = M;
    }
    return best;
}

void orc_alpha_prime(int family, int d, const double* nvec, const double* theta0,
                     const double* h, double alpha, double* aprime, double* qstar)
{
    orc_fam F;
    F.family = family; F.d = d;
    for (int i = 0; i < d; ++i) { F.n[i] = nvec[i]; F.th0[i] = theta0[i]; }
    double logal = log(alpha);
    const double gr = 0.5 * (sqrt(5.0) - 1.0);
    double lo = 1e-12, hi = ORC_SMAX;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double f1 = orc_inv_h(&F, h, logal, exp(x1), NULL);
    double f2 = orc_inv_h(&F, h, logal, exp(x2), NULL);
    while (hi - lo > 1e-15 * fmax(1.0, fabs(hi))) {
        if (f1 >= f2) {
            hi = x2; x2 = x1; f2 = f1;
            x1 = hi - gr * (hi - lo);
            f1 = orc_inv_h(&F, h, logal, exp(x1), NULL);
        } else {
            lo = x1; x1 = x2; f1 = f2;
            x2 = lo + gr * (hi - lo);
            f2 = orc_inv_h(&F, h, logal, exp(x2), NULL);
        }
    }
    double s = 0.5 * (lo + hi);
    double q = exp(s);
    int arg;
    double hv = orc_inv_h(&F, h, logal, q, &arg);
    if (s > ORC_SMAX - 1e-6) {
        double hinf = orc_inv_h_inf(&F, h, logal);
        if (hinf >= hv) { *aprime = exp(hinf); *qstar = INFINITY; return; }
    }
    /* Newton on D(q) = -log alpha + psi(q) - psi(1) - (q-1) psi'(q) = 0,
     * the numerator of dM/dq for the active vertex; D'(q) = -(q-1) psi''(q). */
    double v[4];
    orc_vertex(h, d, arg, v);
    for (int it = 0; it < 3; ++it) {
        double Dq = -logal + orc_psi(&F, v, q) - orc_psi(&F, v, 1.0) - (q - 1.0) * orc_dpsi(&F, v, q);
        double dD = -(q - 1.0) * orc_d2psi(&F, v, q);
        if (!(dD < 0.0)) break;
        double qn = q - Dq / dD;
        if (!(qn > 1.0)) break;
        double hn = orc_inv_h(&F, h, logal, qn, NULL);
        if (hn >= hv - 8e-16 * fmax(1.0, fabs(hv))) { q = qn; hv = fmax(hv, hn); } else break;
    }
    *aprime = exp(hv);
    *qstar = q;
}

/* log-partition of the binomial embedding, for tests: A(theta) = sum n_a softplus(theta_a) */
double orc_log_partition(int family, int d, const double* nvec, const double* theta)
{
    orc_fam F;
    F.family = family; F.d = d;
    for (int i = 0; i < d; ++i) { F.n[i] = nvec[i]; F.th0[i] = 0.0; }
    return orc_A(&F, theta);
}

/* ------------------------------------------------------------------------- */
/* Validation (Alg. validation): CP at the centre, then the optimised          */
/* tilewise Tilt-Bound over the box [theta - h, theta + h].                     */
/* ------------------------------------------------------------------------- */
void orc_validate_bounds(const orc_design* D, int64_t n_tiles, const double* theta,
                         const double* halfwidth, const int32_t* K, const int64_t* R,
                         double delta, double* u0, double* bound, double* qstar)
{
    int d = D->d;
    double nvec[4];
    for (int a = 0; a < d; ++a) nvec[a] = (double)orc_n_max(D);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n_tiles; ++i) {
        double u = orc_cp_upper(R[i], K[i], delta);
        u0[i] = u;
        orc_tilt_bound(0, d, nvec, theta + i * d, halfwidth + i * d, u, bound + i, qstar + i);
    }
}

/* Lower validation bound (Rem. extension-lower with the lower CP estimate):
 * l0 = lower CP of R / K at the centre, lower = optimised lower Tilt-Bound. */
void orc_validate_lower(const orc_design* D, int64_t n_tiles, const double* theta,
                        const double* halfwidth, const int32_t* K, const int64_t* R,
                        double delta, double* l0, double* lower, double* qstar)
{
    int d = D->d;
    double nvec[4];
    for (int a = 0; a < d; ++a) nvec[a] = (double)orc_n_max(D);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n_tiles; ++i) {
        /* 1 - l enters the bound as log(1 - l).  For R > K/2 (l near 1) take
         * 1 - l directly as the upper bound of the K - R failures (binomial
         * symmetry: P(Binom(K, l) >= R) = P(Binom(K, 1 - l) <= K - R)), so that
         * its digits are not lost to the subtraction. */
        double l, la;
        if (2 * R[i] > (int64_t)K[i]) {
            double ap = orc_cp_upper((int64_t)K[i] - R[i], K[i], delta);
            l = 1.0 - ap;
            la = log(ap);
        } else {
            l = orc_cp_lower(R[i], K[i], delta);
            la = log1p(-l);
        }
        l0[i] = l;
        double lb;
        orc_tilt_bound_log(0, d, nvec, theta + i * d, halfwidth + i * d, la, &lb, qstar + i);
        lower[i] = (lb >= 0.0) ? 0.0 : -expm1(lb);
    }
}

/* ------------------------------------------------------------------------- */
/* Randomised test (Sec. 7, after Thm. calibration): the statistic is the pair  */
/* (S, w) with w the sim's tie-break word, the threshold the pair (lambda, c),  */
/* compared lexicographically: reject iff S < lambda, or S = lambda and w < c.  */
/* c = 0 is the plain rule S < lambda.                                          */
/* ------------------------------------------------------------------------- */
static int orc_reject_rand(double S, uint32_t w, double lambda, uint32_t c)
{
    return S < lambda || (S == lambda && w < c);
}

int orc_simulate_rand(const orc_design* D, int64_t n_tiles, const double* theta,
                      const uint32_t* null_mask, const int32_t* K, double lambda, uint32_t c,
                      int64_t* R, int64_t* Xrej, double* score)
{
    int d = D->d;
    int nm = orc_n_max(D);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < n_tiles; ++i) {
        uint32_t t[4] = { 0, 0, 0, 0 };
        for (int a = 0; a < d; ++a) t[a] = orc_threshold(theta[i * d + a]);
        int64_t r = 0, xr[4] = { 0, 0, 0, 0 };
        for (int32_t k = 0; k < K[i]; ++k) {
            int32_t x[12];
            orc_counts(D, t, (uint32_t)k, x);
            double S = orc_statistic(D, x, null_mask[i]);
            if (orc_reject_rand(S, orc_tiebreak(D->seed, (uint32_t)k), lambda, c)) {
                r += 1;
                for (int a = 0; a < d; ++a) xr[a] += x[(D->n_looks - 1) * 4 + a];
            }
        }
        if (R) R[i] = r;
        for (int a = 0; a < d; ++a) {
            if (Xrej) Xrej[i * d + a] = xr[a];
            if (score) score[i * d + a] = (double)xr[a] - (double)nm * orc_sigmoid(theta[i * d + a]) * (double)r;
        }
    }
    return 0;
}

typedef struct {
    double S;
    uint32_t w;
} orc_pair;

static int orc_cmp_pair(const void* a, const void* b)
{
    const orc_pair* x = (const orc_pair*)a;
    const orc_pair* y = (const orc_pair*)b;
    if (x->S < y->S) return -1;
    if (x->S > y->S) return 1;
    return (x->w < y->w) ? -1 : (x->w > y->w) ? 1 : 0;
}

/* Randomised calibration: (lambda_i, c_i) = the k_i-th smallest pair (S, w)
 * of tile i's sims (k_i = floor((K_i + 1) alpha'_i); (-inf, 0) when k_i = 0),
 * and (lambda*, c*) their lexicographic minimum (returned, c* through c_star). */
double orc_calibrate_rand(const orc_design* D, int64_t n_tiles, const double* theta,
                          const double* halfwidth, const uint32_t* null_mask, const int32_t* K,
                          double alpha, double* aprime, int64_t* kidx, double* lambda_tile,
                          uint32_t* c_tile, uint32_t* c_star)
{
    int d = D->d;
    double nvec[4];
    for (int a = 0; a < d; ++a) nvec[a] = (double)orc_n_max(D);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_tiles + 1));
    off[0] = 0;
    for (int64_t i = 0; i < n_tiles; ++i) off[i + 1] = off[i] + K[i];
    double* S = (double*)malloc(sizeof(double) * (size_t)off[n_tiles]);
    orc_simulate(D, n_tiles, theta, null_mask, K, 0.0, NULL, NULL, NULL, S, off);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n_tiles; ++i) {
        double ap, qs;
        orc_alpha_prime(0, d, nvec, theta + i * d, halfwidth + i * d, alpha, &ap, &qs);
        aprime[i] = ap;
        int64_t k = (int64_t)floor(((double)K[i] + 1.0) * ap);
        if (k > K[i]) k = K[i];
        kidx[i] = k;
        orc_pair* P = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)K[i]);
        for (int32_t j = 0; j < K[i]; ++j) {
            P[j].S = S[off[i] + j];
            P[j].w = orc_tiebreak(D->seed, (uint32_t)j);
        }
        qsort(P, (size_t)K[i], sizeof(orc_pair), orc_cmp_pair);
        lambda_tile[i] = (k >= 1) ? P[k - 1].S : -INFINITY;
        c_tile[i] = (k >= 1) ? P[k - 1].w : 0u;
        free(P);
    }
    double lam = INFINITY;
    uint32_t cs = 0u;
    for (int64_t j = 0; j < n_tiles; ++j) {
        if (lambda_tile[j] < lam || (lambda_tile[j] == lam && c_tile[j] < cs)) {
            lam = lambda_tile[j];
            cs = c_tile[j];
        }
    }
    *c_star = cs;
    free(S);
    free(off);
    return lam;
}

/* ------------------------------------------------------------------------- */
/* Calibration (Alg. calibration).                                             */
/* ------------------------------------------------------------------------- */
static int orc_cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* alpha'_i, k_i = floor((K_i + 1) alpha'_i), lambda_i = S_(k_i) (1-indexed,
 * -inf when k_i = 0), and lambda* = min_i lambda_i.  S_work must hold sum K. */
double orc_calibrate(const orc_design* D, int64_t n_tiles, const double* theta,
                     const double* halfwidth, const uint32_t* null_mask, const int32_t* K,
                     double alpha, double* aprime, int64_t* kidx, double* lambda_tile)
{
    int d = D->d;
    double nvec[4];
    for (int a = 0; a < d; ++a) nvec[a] = (double)orc_n_max(D);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_tiles + 1));
    off[0] = 0;
    for (int64_t i = 0; i < n_tiles; ++i) off[i + 1] = off[i] + K[i];
    double* S = (double*)malloc(sizeof(double) * (size_t)off[n_tiles]);
    orc_simulate(D, n_tiles, theta, null_mask, K, 0.0, NULL, NULL, NULL, S, off);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n_tiles; ++i) {
        double ap, qs;
        orc_alpha_prime(0, d, nvec, theta + i * d, halfwidth + i * d, alpha, &ap, &qs);
        aprime[i] = ap;
        int64_t k = (int64_t)floor(((double)K[i] + 1.0) * ap);
        if (k > K[i]) k = K[i];
        kidx[i] = k;
        qsort(S + off[i], (size_t)K[i], sizeof(double), orc_cmp_double);
        lambda_tile[i] = (k >= 1) ? S[off[i] + k - 1] : -INFINITY;
    }
    double lam = INFINITY;
    for (int64_t j = 0; j < n_tiles; ++j)
        if (lambda_tile[j] < lam) lam = lambda_tile[j];
    free(S);
    free(off);
    return lam;
}

/* Score-function adjoint of f_hat = R / K: d f_hat / d theta_a = score_a / K. */
void orc_score_backward(int64_t n_tiles, int d, const double* grad_out, const double* score,
                        const int32_t* K, double* grad_theta)
{
    for (int64_t i = 0; i < n_tiles; ++i)
        for (int a = 0; a < d; ++a)
            grad_theta[i * d + a] = grad_out[i] * score[i * d + a] / (double)K[i];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// bound.cu -- per-tile FP64 bound pass: Clopper-Pearson upper bound, the
// q-optimised tilewise Tilt-Bound, and the calibration target alpha'.
//
// Exponential-family Tilt-Bound (Eq. tilt-bound:exp-fam) for independent
// binomial arms on the logit scale, A(theta) = sum_a n log(1 + e^theta_a):
//   log U(theta0, v, q, a) = (1 - 1/q) log a + sum_a phi_a(q, v_a),
//   phi_a(q, v_a) = psi_a(q v_a)/q - psi_a(v_a),  psi_a(x) = n (sp(theta0_a + x) - sp(theta0_a)).
// A is a sum over arms, so the maximum of log U over the 2^d vertices of the
// box (Thm. 3) is the sum over arms of the larger of the two per-arm terms
// (v_a = +h_a or -h_a): the vertex search costs 2d softplus per q, not d 2^d.
// The optimum over q (Thm. 2: quasi-convex in q) is found by bisection in
// s = log q on the sign of the hand-written derivative
//   d/dq log U = log a / q^2 + sum_a [q v_a psi_a'(q v_a) - psi_a(q v_a)] / q^2.
// The inverted bound (Eq. tilt-bound-inv) uses the same per-arm terms:
//   log U^-1 = q/(q-1) [log alpha - sum_a max_v phi_a],
// maximised over q by bisection on the sign of its derivative.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cse_internal.cuh"

namespace {

#define CSE_HD __host__ __device__

constexpr double SMAX = 40.0;   // search range s = log q in [0, 40]
constexpr int BISECT_F32 = 4;        // FP32 bisection steps on [0, SMAX] before the secant
constexpr int SECANT_F32 = 16;       // cap on FP32 secant (Illinois) steps
constexpr float SECANT_TOL = 1e-5f;  // FP32 stage ends when the bracket is this narrow ...
constexpr float SECANT_STEP = 5e-6f; // ... or when a secant step is this short
constexpr int POLISH_IT = 80;   // cap on FP64 safeguarded-Newton steps

struct ArmGeom {
    double th, h, n, sp0, d1p, d1m;   // d1p/d1m = sp(th +/- h) - sp(th)
};

struct ArmGeomF {
    float th, h, n, sig0, sp0, d1p, d1m;
};

CSE_HD __forceinline__ double softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

CSE_HD __forceinline__ void arm_init(ArmGeom& g, double th, double h, double n)
{
    g.th = th;
    g.h = h;
    g.n = n;
    g.sp0 = softplus(th);
    g.d1p = softplus(th + h) - g.sp0;
    g.d1m = softplus(th - h) - g.sp0;
}

CSE_HD __forceinline__ void arm_init_f(ArmGeomF& f, const ArmGeom& g)
{
    f.th = (float)g.th;
    f.h = (float)g.h;
    f.n = (float)g.n;
    f.sig0 = (float)(1.0 / (1.0 + exp(-g.th)));
    f.sp0 = (float)g.sp0;
    f.d1p = (float)g.d1p;
    f.d1m = (float)g.d1m;
}

// ---------------------------------------------------------------------------
// Per-arm terms.  phi_a(q, v) = n [sp(th + q v) - sp(th)] / q - n [sp(th + v) - sp(th)];
// Phi(q) = sum_a max over v = +-h_a of phi_a; derivatives follow the maximising
// branch (on a tie, the one with the larger first derivative: right derivatives).
// ---------------------------------------------------------------------------

// FP32: the difference sp(th + x) - sp(th) = log1p(sigmoid(th) expm1(x)) for small
// |x| (no cancellation), directly otherwise.
template <int D>
CSE_HD void tilt_phi_f(const ArmGeomF* G, float q, float* Phi, float* dPhi)
{
    constexpr int d = D;
    float P = 0.f, dP = 0.f;
    const float iq = 1.0f / q;
#pragma unroll
    for (int a = 0; a < d; ++a) {
        float best = -INFINITY, bestd = 0.f;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const float v = sg ? -G[a].h : G[a].h;
            const float x = q * v;
            const float y = G[a].th + x;
            const float e = expf(-fabsf(y));
            const float l1e = log1pf(e);
            const float r = e / (1.0f + e);
            float Dd;
            if (fabsf(x) < 0.5f) Dd = log1pf(G[a].sig0 * expm1f(x));
            else Dd = fmaxf(y, 0.0f) + l1e - G[a].sp0;
            const float phi = G[a].n * (Dd * iq - (sg ? G[a].d1m : G[a].d1p));
            // x sigmoid(y) - D without cancellation at large |x|
            float hq;
            if (fabsf(x) < 0.5f) hq = x * ((y >= 0.f) ? 1.0f - r : r) - Dd;
            else hq = (y >= 0.f) ? (G[a].sp0 - G[a].th) - x * r - l1e : x * r - l1e + G[a].sp0;
            const float dphi = G[a].n * hq * iq * iq;
            if (phi > best || (phi == best && dphi > bestd)) {
                best = phi;
                bestd = dphi;
            }
        }
        P += best;
        dP += bestd;
    }
    *Phi = P;
    *dPhi = dP;
}

// FP64 value and first two q-derivatives along the maximising branches.
template <int D>
CSE_HD void tilt_phi(const ArmGeom* G, double q, double* Phi, double* dPhi, double* d2Phi, double* kdist = nullptr)
{
    constexpr int d = D;
    double P = 0.0, dP = 0.0, d2P = 0.0, kd = INFINITY;
    const double iq = 1.0 / q;
#pragma unroll
    for (int a = 0; a < d; ++a) {
        double best = -INFINITY, bestd = 0.0, bestd2 = 0.0;
        double ph[2], dph[2];
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const double v = sg ? -G[a].h : G[a].h;
            const double qv = q * v;
            const double x = G[a].th + qv;
            const double e = exp(-fabs(x));
            const double l1e = log1p(e);
            const double sp = fmax(x, 0.0) + l1e - G[a].sp0;
            const double r = e / (1.0 + e);           // sigmoid(-|x|)
            const double sig = (x >= 0.0) ? 1.0 - r : r;
            const double phi = G[a].n * (sp * iq - (sg ? G[a].d1m : G[a].d1p));
            // q psi'(q v)/n - psi(q v)/n = qv sigmoid(x) - sp(x) + sp(th), written
            // without the cancellation of the two O(qv) terms at large q
            const double hq = (x >= 0.0) ? (G[a].sp0 - G[a].th) - qv * r - l1e : qv * r - l1e + G[a].sp0;
            const double dphi = G[a].n * hq * iq * iq;
            ph[sg] = phi;
            dph[sg] = dphi;
            if (phi > best || (phi == best && dphi > bestd)) {
                best = phi;
                bestd = dphi;
                bestd2 = G[a].n * (v * v * sig * (1.0 - sig) * iq - 2.0 * hq * iq * iq * iq);
            }
        }
        P += best;
        dP += bestd;
        d2P += bestd2;
        // first-order distance in q to the crossing of this arm's two branches
        kd = fmin(kd, fabs(ph[0] - ph[1]) / (fabs(dph[0] - dph[1]) + 1e-300));
    }
    *Phi = P;
    *dPhi = dP;
    if (d2Phi) *d2Phi = d2P;
    if (kdist) *kdist = kd;
}

// lim_{q->inf} Phi(q) = sum_a max(n h_a - n d1p, -n d1m)
template <int D>
CSE_HD double tilt_phi_inf(const ArmGeom* G)
{
    constexpr int d = D;
    double P = 0.0;
    for (int a = 0; a < d; ++a) P += G[a].n * fmax(G[a].h - G[a].d1p, -G[a].d1m);
    return P;
}

// Objective of the q search in s = log q.  kind 0: Tilt-Bound, G(s) = g(e^s),
// g(q) = (1 - 1/q) log a + Phi(q), minimised.  kind 1: inverted bound, negated so
// that it is also minimised: G(s) = -M(e^s), M(q) = q/(q-1) (log alpha - Phi(q)).
// Returns dG/ds (and d2G/ds2, value when asked).
template <int D>
CSE_HD double obj_ds(const ArmGeom* G, int kind, double lc, double s, double* d2, double* val,
                     double* kdist_s = nullptr)
{
    const double q = exp(s);
    double P, dP, d2P, kd;
    tilt_phi<D>(G, q, &P, &dP, &d2P, &kd);
    if (kdist_s) *kdist_s = kd / q;
    double g1, g2, v;
    if (kind == 0) {
        v = (1.0 - 1.0 / q) * lc + P;
        g1 = lc / (q * q) + dP;
        g2 = -2.0 * lc / (q * q * q) + d2P;
    } else {
        const double qm = q - 1.0, B = lc - P;
        v = -(q / qm * B);
        g1 = -(-B / (qm * qm) - q / qm * dP);
        g2 = -(2.0 * B / (qm * qm * qm) + 2.0 * dP / (qm * qm) - q / qm * d2P);
    }
    if (val) *val = v;
    if (d2) *d2 = q * g1 + q * q * g2;
    return q * g1;
}

template <int D>
CSE_HD float obj_ds_f(const ArmGeomF* G, int kind, float lc, float s)
{
    const float q = expf(s);
    float P, dP;
    tilt_phi_f<D>(G, q, &P, &dP);
    if (kind == 0) return q * (lc / (q * q) + dP);
    const float qm = q - 1.0f;
    // sign of -dM/dq: -(log alpha - Phi) ... expressed without dividing by (q-1)^2
    return -(-(lc - P) - q * qm * dP);
}

// Coordinates in which the FP32 secant interpolates G'(s) linearly.  With Phi
// linear in q (its first-order form for small q h), kind 0 has dG/dq = G'(s)/q
// affine in 1/q^2, and kind 1 has the sign function of obj_ds_f affine in
// (q - 1)^2: so y = G'(s) e^{-s} against t = e^{-2s} for kind 0, and y = that
// function against t = (e^s - 1)^2 for kind 1.  The secant then converges in a
// few steps.
CSE_HD __forceinline__ void secant_point(int kind, float s, float g, float* t, float* y)
{
    if (kind == 0) {
        const float e = expf(-s);
        *t = e * e;
        *y = g * e;
    } else {
        const float e = expm1f(s);
        *t = e * e;
        *y = g;
    }
}

CSE_HD __forceinline__ float secant_s(int kind, float t)
{
    return kind == 0 ? -0.5f * logf(t) : log1pf(sqrtf(t));
}

// Minimiser of the quasi-convex G over s in [0, SMAX].  FP32 stage: the sign of
// G' at s = 0, a few bisection steps, then a bracketing secant (Illinois: the
// stale end's value is halved when the same end moves twice running) in the
// coordinates of secant_point, down to ~1e-5 in s.  FP64 stage: safeguarded
// Newton from the secant's last point refines it (bisection fallback).
// Returns s*, *val = G(s*).
template <int D>
CSE_HD double q_search(const ArmGeom* G, int kind, double lc, double* val)
{
    constexpr int d = D;
    ArmGeomF Gf[D];
#pragma unroll
    for (int a = 0; a < d; ++a) arm_init_f(Gf[a], G[a]);
    float flo = 0.0f, fhi = (float)SMAX, sx = NAN;
    const float lcf = (float)lc;
    const float f0 = obj_ds_f<D>(Gf, kind, lcf, 0.0f);
    const bool at_one = !(f0 < 0.0f);
    if (at_one) {
        // G' not negative at q = 1: the boundary case below decides (FP64)
        fhi = (float)SMAX * 0x1p-22f;
    } else {
        float fa = f0, fb = NAN;
        for (int it = 0; it < BISECT_F32; ++it) {
            const float mid = 0.5f * (flo + fhi);
            const float fm = obj_ds_f<D>(Gf, kind, lcf, mid);
            if (fm < 0.0f) { flo = mid; fa = fm; } else { fhi = mid; fb = fm; }
        }
        float ta, ya, tb, yb;
        secant_point(kind, flo, fa, &ta, &ya);
        secant_point(kind, fhi, fb, &tb, &yb);
        int side = 0;
        for (int it = 0; it < SECANT_F32; ++it) {
            float xn = 0.5f * (flo + fhi);   // bisection while G'(fhi) is unknown
            if (yb == yb) {
                const float xs = secant_s(kind, ta - ya * ((tb - ta) / (yb - ya)));
                if (xs == xs) {
                    if (!(xs > flo && xs < fhi)) {   // the root is within rounding of an end
                        sx = (xs < xn) ? flo : fhi;
                        break;
                    }
                    if (sx == sx && fabsf(xs - sx) <= SECANT_STEP) {
                        sx = xs;
                        break;
                    }
                    xn = xs;
                }
            }
            const float fx = obj_ds_f<D>(Gf, kind, lcf, xn);
            float tx, yx;
            secant_point(kind, xn, fx, &tx, &yx);
            sx = xn;
            if (fx < 0.0f) {
                flo = xn; ta = tx; ya = yx;
                if (side < 0) yb *= 0.5f;
                side = -1;
            } else {
                fhi = xn; tb = tx; yb = yx;
                if (side > 0) ya *= 0.5f;
                side = 1;
            }
            if (fhi - flo <= SECANT_TOL) break;
        }
    }
    if (!(sx == sx)) sx = 0.5f * (flo + fhi);
    // minimum at the boundary q = 1 (the objective is quasi-convex in q, Thm. 2):
    // G' was not negative at s = 0 in FP32 and is not in FP64 either.  For the
    // Tilt-Bound the value at q = 1 is 0 exactly (U = 1).
    if (kind == 0 && at_one) {
        double v0;
        if (!(obj_ds<D>(G, kind, lc, 0.0, nullptr, &v0) < 0.0)) {
            *val = v0;
            return 0.0;
        }
    }
    // fast path: Newton from the FP32 estimate; at a smooth optimum two FP64
    // evaluations reach ~1e-20 in s, and the value at the last evaluated point is
    // exact to second order
    double s = (double)sx;
    {
        // one FP64 evaluation: at a smooth optimum a Newton step from the FP32
        // estimate and the second-order Taylor value are exact to O(step^3)
        double d2, v, kd;
        const double g1 = obj_ds<D>(G, kind, lc, s, &d2, &v, &kd);
        if (d2 > 0.0) {
            const double step = g1 / d2;
            if (fabs(step) <= 4e-5 && kd > 16.0 * fabs(step) + 1e-6 && s - step > 0.0 && s - step < SMAX) {
                *val = v - 0.5 * g1 * step;
                return s - step;
            }
        }
    }
    {
        // Newton steps may leave the FP32 bracket (its derivative's sign can be
        // wrong close to the root) by up to 1e-2 in s; kinks go to the robust path
        const double flo_m = fmax(0.0, (double)flo - 1e-2), fhi_m = fmin(SMAX, (double)fhi + 1e-2);
        for (int it = 0; it < 6; ++it) {
            double d2, v;
            const double g1 = obj_ds<D>(G, kind, lc, s, &d2, &v);
            if (g1 == 0.0) {
                *val = v;
                return s;
            }
            if (!(d2 > 0.0)) break;
            const double step = g1 / d2;
            if (fabs(step) <= 1e-8) {
                *val = v;
                return s - step;
            }
            const double sn = s - step;
            if (!(sn > flo_m && sn < fhi_m)) break;
            s = sn;
        }
    }
    // robust path (kinks of the piecewise-smooth objective, or an FP32 bracket
    // spoilt by rounding): verified bracket, safeguarded Newton with bisection
    double lo = fmax(0.0, (double)flo - 1e-3), hi = fmin(SMAX, (double)fhi + 1e-3);
    if (lo > 0.0 && !(obj_ds<D>(G, kind, lc, lo, nullptr, nullptr) < 0.0)) lo = 0.0;
    if (kind == 0 && lo == 0.0 && !at_one) {   // the boundary test above, for a spoilt bracket
        double v0;
        if (!(obj_ds<D>(G, kind, lc, 0.0, nullptr, &v0) < 0.0)) {
            *val = v0;
            return 0.0;
        }
    }
    if (hi < SMAX && obj_ds<D>(G, kind, lc, hi, nullptr, nullptr) < 0.0) hi = SMAX;
    s = fmin(fmax((double)sx, lo), hi);
    for (int it = 0; it < POLISH_IT; ++it) {
        double d2;
        const double g1 = obj_ds<D>(G, kind, lc, s, &d2, nullptr);
        if (g1 == 0.0) break;
        // a Newton step below 1e-11 at a smooth point: the value is then exact to
        // ~d2 1e-22, well past FP64 (at a kink g1 does not shrink and bisection runs on)
        if (d2 > 0.0 && fabs(g1 / d2) <= 1e-11 * fmax(1.0, fabs(s))) {
            s -= g1 / d2;
            break;
        }
        if (g1 < 0.0) lo = s; else hi = s;
        if (hi - lo <= 1e-15 * fmax(1.0, hi)) break;
        double sn = s - g1 / d2;
        if (!(d2 > 0.0) || !(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
        if (fabs(sn - s) <= 4e-16 * fmax(1.0, fabs(s))) {
            s = sn;
            break;
        }
        s = sn;
    }
    obj_ds<D>(G, kind, lc, s, nullptr, val);
    return s;
}

// Plain form of the q search: FP64 bisection on the sign of G' over [0, SMAX]
// (64 halvings), no FP32 stage.  Same optimum, more FP64 work.
template <int D>
CSE_HD double q_search_plain(const ArmGeom* G, int kind, double lc, double* val)
{
    double lo = 0.0, hi = SMAX;
    for (int it = 0; it < 64; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (obj_ds<D>(G, kind, lc, mid, nullptr, nullptr) < 0.0) lo = mid; else hi = mid;
    }
    const double s = 0.5 * (lo + hi);
    obj_ds<D>(G, kind, lc, s, nullptr, val);
    return s;
}

// log inf_q max_v U(theta0, v, q, a) from log a (a = 1 - l keeps its digits as
// log1p(-l)); *qstar the minimiser.  q = 1 gives U = 1 exactly, so the result
// is at most 0.
template <int D, bool PLAIN = false>
CSE_HD double tilt_bound_log_la(const ArmGeom* G, double la, double* qstar)
{
    if (la >= 0.0) {
        *qstar = 1.0;
        return 0.0;
    }
    if (la == -INFINITY) {
        *qstar = INFINITY;
        return -INFINITY;
    }
    double val;
    const double s = PLAIN ? q_search_plain<D>(G, 0, la, &val) : q_search<D>(G, 0, la, &val);
    if (s > SMAX - 1e-6) {
        const double vinf = la + tilt_phi_inf<D>(G);
        if (vinf <= val) {
            *qstar = INFINITY;
            return vinf;
        }
    }
    if (val > 0.0) {
        *qstar = 1.0;
        return 0.0;
    }
    *qstar = exp(s);
    return val;
}

// inf_q max_v U(theta0, v, q, a); returns log bound, *qstar.
template <int D, bool PLAIN = false>
CSE_HD double tilt_bound_log(const ArmGeom* G, double a, double* qstar)
{
    if (a >= 1.0) {
        *qstar = 1.0;
        return 0.0;
    }
    if (!(a > 0.0)) {
        *qstar = INFINITY;
        return -INFINITY;
    }
    return tilt_bound_log_la<D, PLAIN>(G, log(a), qstar);
}

// sup_q min_v U^-1(theta0, v, q, alpha); returns log alpha', *qstar.
template <int D, bool PLAIN = false>
CSE_HD double alpha_prime_log(const ArmGeom* G, double alpha, double* qstar)
{
    const double lal = log(alpha);
    double val;
    const double s = PLAIN ? q_search_plain<D>(G, 1, lal, &val) : q_search<D>(G, 1, lal, &val);
    val = -val;
    if (s > SMAX - 1e-6) {
        const double vinf = lal - tilt_phi_inf<D>(G);
        if (vinf >= val) {
            *qstar = INFINITY;
            return vinf;
        }
    }
    *qstar = exp(s);
    return val;
}

// ---------------------------------------------------------------------------
// Clopper-Pearson (Eq. clopper-pearson:def): u with P(Binom(N, u) <= R) = delta,
// i.e. I_{1-u}(N - R, R + 1) = delta.  Newton in log space on the regularised
// incomplete beta function (continued fraction times its prefactor): an FP32
// solve to ~1e-6, then FP64 steps until the step is below 1e-9 relative
// (quadratic convergence leaves ~1e-18).
// ---------------------------------------------------------------------------

// Stirling-series remainder lgamma(z) - [(z - 1/2) log z - z + log(2 pi)/2], z >= 10.
CSE_HD __forceinline__ double stirling_rem(double z)
{
    const double r = 1.0 / z, r2 = r * r;
    return r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0 - r2 * (1.0 / 1680.0 - r2 / 1188.0))));
}

CSE_HD __forceinline__ float stirling_rem_f(float z)
{
    const float r = 1.0f / z, r2 = r * r;
    return r * (1.0f / 12.0f - r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
}

// lgamma of a positive integer below 19: log of the exactly representable factorial
CSE_HD __forceinline__ double lgamma_small_int(double z)
{
    double f = 1.0;
    for (int k = 2; k < (int)z; ++k) f *= (double)k;
    return log(f);
}

// log(x^a y^b / B(a, b)) for integer a, b >= 1, with lx = log x, ly = log y
// (y = 1 - x) and e = x (a + b) - a supplied accurately by the caller.
CSE_HD double log_bpre(double a, double b, double lx, double ly, double e)
{
    const double L2PI = 1.8378770664093454836;
    if (a >= 10.0 && b >= 10.0) {
        return a * log1p(e / a) + b * log1p(-e / b) + 0.5 * log(a * b / (a + b)) - 0.5 * L2PI
               - (stirling_rem(a) + stirling_rem(b) - stirling_rem(a + b));
    }
    if (b >= 10.0) {   // small a: lgamma(a+b) - lgamma(b) by the Stirling difference
        return a * lx + b * ly - lgamma_small_int(a) + a * log(a + b) + (b - 0.5) * log1p(a / b) - a
               + stirling_rem(a + b) - stirling_rem(b);
    }
    if (a >= 10.0) {
        return a * lx + b * ly - lgamma_small_int(b) + b * log(a + b) + (a - 0.5) * log1p(b / a) - b
               + stirling_rem(a + b) - stirling_rem(a);
    }
    return a * lx + b * ly - lgamma_small_int(a) - lgamma_small_int(b) + lgamma_small_int(a + b);
}

CSE_HD float log_bpre_f(float a, float b, float lx, float ly, float e)
{
    if (a >= 10.0f && b >= 10.0f) {
        return a * log1pf(e / a) + b * log1pf(-e / b) + 0.5f * logf(a * b / (a + b)) - 0.9189385332f
               - (stirling_rem_f(a) + stirling_rem_f(b) - stirling_rem_f(a + b));
    }
    return a * lx + b * ly - lgammaf(a) - lgammaf(b) + lgammaf(a + b);
}

// Continued fraction 1/(1 + d1/(1 + d2/(1 + ...))) of I_x(a, b), with
// d_{2m+1} = -(a+m)(a+b+m)x / ((a+2m)(a+2m+1)), d_{2m} = m(b-m)x / ((a+2m-1)(a+2m)).
// FP64, division-free: three-term recurrences of the equivalent fraction whose
// partial numerators / denominators are the polynomials p, q of d = p/q, rescaled
// by exact powers of two; one division per convergence check.
CSE_HD double beta_cf(double a, double b, double x)
{
    // d_{2m+1} = p_odd / q_odd, d_{2m} = p_even / q_even; the numerator and
    // denominator polynomials are advanced by their differences in m
    double po_f = a * (a + b);             // (a+m)(a+b+m) at m = 0
    double po_df = 2.0 * a + b + 1.0;      // its first difference at m = 0
    double qo = a * (a + 1.0);             // (a+2m)(a+2m+1) at m = 0
    double qo_d = 4.0 * a + 6.0;           // first difference (second difference 8)
    double pe_f = b - 1.0;                 // m (b-m) at m = 1
    double pe_df = b - 3.0;                // first difference at m = 1 (second difference -2)
    double qe = (a + 1.0) * (a + 2.0);     // (a+2m-1)(a+2m) at m = 1
    double qe_d = 4.0 * a + 10.0;          // first difference (second difference 8)
    double Am2 = 0.0, Am1 = 1.0, Bm2 = 1.0, Bm1 = 1.0;   // A_0, A_1, B_0, B_1
    double qprev = 1.0, f_old = 1.0;
    const double BIG = 0x1p600, SMALL = 0x1p-600;
    for (int k = 2; k < 4000; ++k) {
        double p, q;
        if (k & 1) {                       // level k uses d_{k-1}, k-1 even
            p = pe_f * x;
            q = qe;
            pe_f += pe_df;
            pe_df -= 2.0;
            qe += qe_d;
            qe_d += 8.0;
        } else {                           // k-1 odd
            p = -po_f * x;
            q = qo;
            po_f += po_df;
            po_df += 2.0;
            qo += qo_d;
            qo_d += 8.0;
        }
        const double an = qprev * p;
        const double A = q * Am1 + an * Am2;
        const double B = q * Bm1 + an * Bm2;
        Am2 = Am1;
        Am1 = A;
        Bm2 = Bm1;
        Bm1 = B;
        qprev = q;
        if (fabs(Bm1) > BIG) {             // exact rescaling by a power of two
            Am2 *= SMALL;
            Am1 *= SMALL;
            Bm2 *= SMALL;
            Bm1 *= SMALL;
        }
        if ((k & 7) == 0) {
            const double f = Am1 / Bm1;
            if (fabs(f - f_old) <= 1e-14 * fabs(f)) return f;
            f_old = f;
        }
    }
    return Am1 / Bm1;
}

// Quotient for the FP32 search stage, which needs ~1e-6: the device uses the
// two-instruction approximate division (2 ulp).
CSE_HD __forceinline__ float fdiv_fast(float x, float y)
{
#ifdef __CUDA_ARCH__
    return __fdividef(x, y);
#else
    return x / y;
#endif
}

// FP32 modified Lentz evaluation of the same fraction (start of the solve).
CSE_HD float beta_cf_f(float a, float b, float x)
{
    const float TINY = 1e-30f;
    const float qab = a + b, qap = a + 1.0f, qam = a - 1.0f;
    float c = 1.0f, dd = 1.0f - fdiv_fast(qab * x, qap);
    if (fabsf(dd) < TINY) dd = TINY;
    dd = fdiv_fast(1.0f, dd);
    float h = dd;
    for (int m = 1; m <= 300; ++m) {
        const float m2 = 2.0f * m;
        float aa = fdiv_fast(m * (b - m) * x, (qam + m2) * (a + m2));
        dd = 1.0f + aa * dd;
        if (fabsf(dd) < TINY) dd = TINY;
        c = 1.0f + fdiv_fast(aa, c);
        if (fabsf(c) < TINY) c = TINY;
        dd = fdiv_fast(1.0f, dd);
        h *= dd * c;
        aa = -fdiv_fast((a + m) * (qab + m) * x, (a + m2) * (qap + m2));
        dd = 1.0f + aa * dd;
        if (fabsf(dd) < TINY) dd = TINY;
        c = 1.0f + fdiv_fast(aa, c);
        if (fabsf(c) < TINY) c = TINY;
        dd = fdiv_fast(1.0f, dd);
        const float del = dd * c;
        h *= del;
        // the FP32 phase needs ~1e-6: a 1-ulp test may never be met under FMA rounding
        if (fabsf(del - 1.0f) <= 1e-6f) break;
    }
    return h;
}

// log P(Binom(N, u) <= R) = log I_{1-u}(b, a) and log pdf of Beta(a, b) at u,
// a = R + 1, b = N - R.  The prefactor is symmetric in (a, u) <-> (b, 1 - u).
CSE_HD double log_binom_cdf(double a, double b, double u, double* lpdf)
{
    const double lu = log(u), l1u = log1p(-u);
    const double e = fma(u, a + b, -a);   // u (a+b) - a
    const double lp = log_bpre(a, b, lu, l1u, e);
    *lpdf = lp - lu - l1u;
    if (u >= (a + 1.0) / (a + b + 2.0)) return lp + log(beta_cf(b, a, 1.0 - u)) - log(b);
    return log1p(-exp(lp) * beta_cf(a, b, u) / a);
}

CSE_HD float log_binom_cdf_f(float a, float b, float u, float* lpdf)
{
    const float lu = logf(u), l1u = log1pf(-u);
    const float e = fmaf(u, a + b, -a);
    const float lp = log_bpre_f(a, b, lu, l1u, e);
    *lpdf = lp - lu - l1u;
    if (u >= (a + 1.0f) / (a + b + 2.0f)) return lp + logf(beta_cf_f(b, a, 1.0f - u)) - logf(b);
    return log1pf(-expf(lp) * beta_cf_f(a, b, u) / a);
}

// Small R: log P(Binom(N, u) <= R) = N log(1-u) + log sum_{j<=R} C(N,j) w^j,
// w = u / (1-u), by the term recurrence t_{j+1} = t_j (N-j) w / (j+1); the
// Beta(R+1, N-R) log density at u is log((N-R) t_R) + (N-1) log(1-u) + ... .
constexpr int64_t CP_SMALL_R = 40;
CSE_HD double log_binom_cdf_small(int64_t R, int64_t N, double u, double* lpdf)
{
    const double l1u = log1p(-u);
    const double w = u / (1.0 - u);
    double t = 1.0, sum = 1.0;
    for (int64_t j = 0; j < R; ++j) {
        t *= (double)(N - j) * w / (double)(j + 1);
        sum += t;
    }
    const double base = (double)N * l1u;
    *lpdf = log((double)(N - R) * t) + base - l1u;
    return base + log(sum);
}

// Plain form: FP64 Newton from the normal-approximation start, no FP32 stage.
CSE_HD double cp_upper_plain(int64_t R, int64_t N, double delta)
{
    if (R >= N) return 1.0;
    if (R <= 0) return -expm1(log(delta) / (double)N);
    const double a = (double)R + 1.0, b = (double)(N - R);
    const double ld = log(delta);
    const double mean = a / (a + b);
    const double sd = sqrt(a * b / ((a + b) * (a + b) * (a + b + 1.0)));
    double u = fmin(mean + 2.5 * sd, 0.5 * (mean + 1.0));
    const bool small = R < CP_SMALL_R && N - R > CP_SMALL_R;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 100; ++it) {
        double lpdf;
        const double lF = small ? log_binom_cdf_small(R, N, u, &lpdf) : log_binom_cdf(a, b, u, &lpdf);
        const double f = lF - ld;
        const double nstep = f / (-exp(lpdf - lF));
        if (fabs(nstep) <= 4e-16 * u) break;
        if (f > 0.0) lo = u; else hi = u;
        double un = u - nstep;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        u = un;
    }
    return u;
}

// FP32 f(u) = log P(Binom(N,u) <= R) - log delta (the FP32 search stage)
CSE_HD float cp_f32(int64_t R, int64_t N, float u, float ldf, float* lpdf)
{
    const bool small = R < CP_SMALL_R && N - R > CP_SMALL_R;
    if (small) {
        const float l1u = log1pf(-u), w = u / (1.0f - u);
        float t = 1.0f, sum = 1.0f;
        for (int j = 0; j < (int)R; ++j) {
            t *= fdiv_fast((float)(N - j) * w, (float)(j + 1));
            sum += t;
        }
        const float base = (float)N * l1u;
        if (lpdf) *lpdf = logf((float)(N - R) * t) + base - l1u;
        return base + logf(sum) - ldf;
    }
    float lp;
    const float lF = log_binom_cdf_f((float)R + 1.0f, (float)(N - R), u, &lp);
    if (lpdf) *lpdf = lp;
    return lF - ldf;
}

// FP64 stage from an estimate u: Halley steps on phi(u) = log F(u) - log delta,
// phi' = -pdf/F, phi'' = -(pdf/F) ((a-1)/u - (b-1)/(1-u)) - (pdf/F)^2.  From an
// FP32-accurate estimate one step leaves an error of order step^3.
CSE_HD double cp_finish_fp64(int64_t R, int64_t N, double delta, double u)
{
    const double a = (double)R + 1.0, b = (double)(N - R);
    const double ld = log(delta);
    const bool small = R < CP_SMALL_R && N - R > CP_SMALL_R;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
        double lpdf;
        const double lF = small ? log_binom_cdf_small(R, N, u, &lpdf) : log_binom_cdf(a, b, u, &lpdf);
        const double f = lF - ld;
        if (f == 0.0) break;
        const double r = exp(lpdf - lF);
        const double p1 = -r;
        const double p2 = -r * ((a - 1.0) / u - (b - 1.0) / (1.0 - u)) - r * r;
        const double den = 2.0 * p1 * p1 - f * p2;
        const double du = (den != 0.0) ? -2.0 * f * p1 / den : -f / p1;
        if (fabs(du) <= 4e-16 * u) break;   // converged to rounding
        if (f > 0.0) lo = u; else hi = u;
        double un = u + du;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        const double step = fabs(un - u);
        u = un;
        if (step <= 3e-6 * fmin(u, 1.0 - u) || hi - lo <= 4e-16 * hi) break;
    }
    return u;
}

CSE_HD double cp_upper(int64_t R, int64_t N, double delta)
{
    if (R >= N) return 1.0;
    if (R <= 0) return -expm1(log(delta) / (double)N);
    const double a = (double)R + 1.0, b = (double)(N - R);
    const double mean = a / (a + b);
    const double sd = sqrt(a * b / ((a + b) * (a + b) * (a + b + 1.0)));
    double u = fmin(mean + 2.5 * sd, 0.5 * (mean + 1.0));
    // FP32 stage: safeguarded Newton
    {
        const float ldf = (float)log(delta);
        float uf = (float)u, lof = 0.0f, hif = 1.0f;
        for (int it = 0; it < 16; ++it) {
            float lpdf;
            const float f = cp_f32(R, N, uf, ldf, &lpdf);
            if (f > 0.0f) lof = uf; else hif = uf;
            const float dlF = -expf(lpdf - (f + ldf));
            float un = uf - f / dlF;
            if (!(un > lof && un < hif)) un = 0.5f * (lof + hif);
            const bool done = fabsf(un - uf) <= 1e-6f * uf;
            uf = un;
            if (done) break;
        }
        if (uf > 0.0f && uf < 1.0f) u = (double)uf;
    }
    return cp_finish_fp64(R, N, delta, u);
}

// Search interval of the cooperative FP32 stage: lo = 0 and hi = 1 or 14 standard
// deviations above the mean of Beta(R+1, N-R) (a log-concave law, so F(hi) is
// below e^-13 there).
CSE_HD void cp_interval(int64_t R, int64_t N, float* lo, float* hi)
{
    const float a = (float)R + 1.0f, b = (float)(N - R), s = a + b;
    const float mean = a / s;
    const float sd = sqrtf(a * b / (s * s * (s + 1.0f)));
    *lo = 0.0f;
    *hi = fminf(1.0f, mean + 14.0f * sd + 4.0f / s);
}

// Point j of one round of the cooperative search: 32 interior points split
// (lo, hi) into 33 equal parts.
CSE_HD void cp_round_points(float lo, float hi, int j, float* uj)
{
    *uj = lo + (hi - lo) * ((float)(j + 1) / 33.0f);
}

// ---------------------------------------------------------------------------
// Warp-wide FP64 evaluation of the Clopper-Pearson equation.  On this part an
// FP64 warp instruction costs the same pipe time however many lanes it has
// active, so the per-key FP64 work is spread over the 32 lanes:
//  * the continued fraction as a composition of linear fractional maps, i.e. a
//    product of 2x2 matrices (associative): each lane multiplies 8 consecutive
//    levels, a 5-step shuffle tree forms the ordered product, and the product
//    of the first 16 lanes gives, for free, the convergent at half the depth,
//    which is the convergence test;
//  * the small-R binomial sum as a warp prefix product of term ratios.
// Every lane returns the same value.
// ---------------------------------------------------------------------------
struct Mat2 {
    double m00, m01, m10, m11;
};

__device__ __forceinline__ Mat2 mat2_mul(const Mat2& A, const Mat2& B)
{
    return {fma(A.m00, B.m00, A.m01 * B.m10), fma(A.m00, B.m01, A.m01 * B.m11),
            fma(A.m10, B.m00, A.m11 * B.m10), fma(A.m10, B.m01, A.m11 * B.m11)};
}

__device__ __forceinline__ int exp_field(double x)
{
    return (__double2hiint(x) >> 20) & 0x7ff;
}

// Scales by the power of two that brings the largest entry into [1, 2): exact,
// and the convergents are ratios of entries, so they are unchanged.
__device__ __forceinline__ Mat2 mat2_norm(Mat2 A)
{
    int e = max(max(exp_field(A.m00), exp_field(A.m01)), max(exp_field(A.m10), exp_field(A.m11)));
    e = min(max(e, 1), 2045);
    const double sc = __hiloint2double((2046 - e) << 20, 0);
    A.m00 *= sc;
    A.m01 *= sc;
    A.m10 *= sc;
    A.m11 *= sc;
    return A;
}

__device__ __forceinline__ Mat2 mat2_shfl_down(const Mat2& A, int s)
{
    return {__shfl_down_sync(0xffffffffu, A.m00, s), __shfl_down_sync(0xffffffffu, A.m01, s),
            __shfl_down_sync(0xffffffffu, A.m10, s), __shfl_down_sync(0xffffffffu, A.m11, s)};
}

__device__ __forceinline__ Mat2 mat2_bcast(const Mat2& A, int src)
{
    return {__shfl_sync(0xffffffffu, A.m00, src), __shfl_sync(0xffffffffu, A.m01, src),
            __shfl_sync(0xffffffffu, A.m10, src), __shfl_sync(0xffffffffu, A.m11, src)};
}

// Right-multiplies C by the map t -> d / (1 + t), d = p / q, as the matrix
// [[0, p], [q, q]] (a common factor q does not change the map).
__device__ __forceinline__ void cf_level(Mat2& C, double p, double q)
{
    const double c00 = C.m00, c10 = C.m10;
    C.m00 = C.m01 * q;
    C.m01 = fma(c00, p, C.m01 * q);
    C.m10 = C.m11 * q;
    C.m11 = fma(c10, p, C.m11 * q);
}

// The fraction 1/(1 + d1/(1 + d2/(1 + ...))) of I_x(a, b) (same d_j as beta_cf),
// as the composition of the maps t -> 1/(1 + t) (level 0) and t -> d_j/(1 + t)
// applied to t = 0: with Q = N_0 N_1 ... N_n, the n-level convergent is
// Q01 / Q11, a ratio of two entries of one column, and rescaling Q by a power
// of two leaves it exact.  Lane chunk g holds levels 8g .. 8g+7, so level 0
// is multiplied first, in sequence, where the leading partial fractions
// cancel (d_{2m+1} near -1 for x near the mean).  For integer b the fraction
// ends at d_{2b} = 0; the levels past it are left out.
__device__ double beta_cf_warp(double a, double b, double x, int lane)
{
    constexpr int PAIRS = 4;   // levels (d_{2m}, d_{2m+1}) per lane per pass
    Mat2 P = {1.0, 0.0, 0.0, 1.0};
    double f = 0.0;
    for (int pass = 0; pass < 16; ++pass) {   // 256 levels a pass
        Mat2 C = {1.0, 0.0, 0.0, 1.0};
        const double g = (double)(pass * 32 + lane);
#pragma unroll
        for (int i = 0; i < PAIRS; ++i) {
            const double m = fma((double)PAIRS, g, (double)i);
            if (m < b) {
                const double a2m = fma(2.0, m, a);
                if (m > 0.0)   // d_{2m} = m(b-m) x / ((a+2m-1)(a+2m))
                    cf_level(C, (m * (b - m)) * x, (a2m - 1.0) * a2m);
                else           // level 0: t -> 1/(1 + t)
                    C = {0.0, 1.0, 1.0, 1.0};
                const double am = a + m;   // d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1))
                cf_level(C, -(am * (am + b)) * x, a2m * (a2m + 1.0));
            }
        }
        C = mat2_norm(C);
        Mat2 half = C;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {   // lane 0 ends with lanes 0..2sh-1
            C = mat2_norm(mat2_mul(C, mat2_shfl_down(C, sh)));
            if (sh == 8) half = C;
        }
        const Mat2 Pm = mat2_mul(P, mat2_bcast(half, 0));
        P = mat2_norm(mat2_mul(P, mat2_bcast(C, 0)));
        const double f_mid = Pm.m01 / Pm.m11;
        f = P.m01 / P.m11;
        if (fabs(f - f_mid) <= 1e-14 * fabs(f)) break;
    }
    return f;
}

// The logarithms and Stirling remainders of log_bpre, one per lane: lane k
// evaluates term k (the same function of the same argument as the serial
// form, so the values agree bit for bit) and every lane receives all of them.
//   0 log u, 1 log1p(-u), 2 log1p(e/a), 3 log1p(-e/b), 4 log(ab/(a+b)),
//   5 log(a+b), 6 log1p(a/b), 7 log1p(b/a), 8 log b, 9..11 stirling_rem(a, b, a+b)
constexpr int N_PREFIX_TERMS = 12;
__device__ void prefix_terms_warp(double a, double b, double u, int lane, double* T)
{
    const double e = fma(u, a + b, -a);
    double num = 1.0, den = 1.0;
    int kind = 0;   // 0 log(num/den), 1 log1p(num/den), 2 Stirling remainder of den, 3 none
    switch (lane) {
    case 0: num = u; break;
    case 1: num = -u; kind = 1; break;
    case 2: num = e; den = a; kind = 1; break;
    case 3: num = -e; den = b; kind = 1; break;
    case 4: num = a * b; den = a + b; break;
    case 5: num = a + b; break;
    case 6: num = a; den = b; kind = 1; break;
    case 7: num = b; den = a; kind = 1; break;
    case 8: num = b; break;
    case 9: den = a; kind = 2; break;
    case 10: den = b; kind = 2; break;
    case 11: den = a + b; kind = 2; break;
    default: kind = 3;
    }
    const double q = num / den;
    double v = 0.0;
    if (kind == 0) {
        v = log(q);
    } else if (kind == 1) {
        v = log1p(q);
    } else if (kind == 2) {   // stirling_rem with r = 1/z
        const double r2 = q * q;
        v = q * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0 - r2 * (1.0 / 1680.0 - r2 / 1188.0))));
    }
#pragma unroll
    for (int k = 0; k < N_PREFIX_TERMS; ++k) T[k] = __shfl_sync(0xffffffffu, v, k);
}

// log_bpre from the lane-evaluated terms (same formulas, same operation order).
__device__ double log_bpre_terms(double a, double b, const double* T)
{
    const double L2PI = 1.8378770664093454836;
    if (a >= 10.0 && b >= 10.0) return a * T[2] + b * T[3] + 0.5 * T[4] - 0.5 * L2PI - (T[9] + T[10] - T[11]);
    if (b >= 10.0) return a * T[0] + b * T[1] - lgamma_small_int(a) + a * T[5] + (b - 0.5) * T[6] - a + T[11] - T[10];
    if (a >= 10.0) return a * T[0] + b * T[1] - lgamma_small_int(b) + b * T[5] + (a - 0.5) * T[7] - b + T[11] - T[9];
    return a * T[0] + b * T[1] - lgamma_small_int(a) - lgamma_small_int(b) + lgamma_small_int(a + b);
}

__device__ double log_binom_cdf_warp(double a, double b, double u, double* lpdf, int lane)
{
    double T[N_PREFIX_TERMS];
    prefix_terms_warp(a, b, u, lane, T);
    const double lp = log_bpre_terms(a, b, T);
    *lpdf = lp - T[0] - T[1];
    if (u >= (a + 1.0) / (a + b + 2.0)) return lp + log(beta_cf_warp(b, a, 1.0 - u, lane)) - T[8];
    return log1p(-exp(lp) * beta_cf_warp(a, b, u, lane) / a);
}

// Small R: the terms t_j = prod_{i<=j} r_i, r_i = (N-i+1) w / i, by a warp
// prefix product; their sum by a butterfly (bitwise equal in every lane).
__device__ double log_binom_cdf_small_warp(int64_t R, int64_t N, double u, double* lpdf, int lane)
{
    const double l1u = log1p(-u);
    const double w = u / (1.0 - u);
    double carry = 1.0, sum = 0.0, tR = 1.0;
    for (int64_t j0 = 1; j0 <= R; j0 += 32) {
        const int64_t j = j0 + lane;
        double t = (j <= R) ? (double)(N - j + 1) * w / (double)j : 1.0;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {
            const double o = __shfl_up_sync(0xffffffffu, t, sh);
            if (lane >= sh) t *= o;
        }
        t *= carry;
        double ts = (j <= R) ? t : 0.0;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) ts += __shfl_xor_sync(0xffffffffu, ts, sh);
        sum += ts;
        const int64_t last = R - j0;   // lane holding j = R, when in this pass
        if (last < 32) tR = __shfl_sync(0xffffffffu, t, (int)last);
        carry = __shfl_sync(0xffffffffu, t, 31);
    }
    sum += 1.0;
    const double base = (double)N * l1u;
    const double lg = log(lane == 0 ? (double)(N - R) * tR : sum);   // two logarithms, two lanes
    *lpdf = __shfl_sync(0xffffffffu, lg, 0) + base - l1u;
    return base + __shfl_sync(0xffffffffu, lg, 1);
}

// cp_finish_fp64 with the warp-wide evaluation (all lanes call it together).
__device__ double cp_finish_warp(int64_t R, int64_t N, double delta, double u, int lane)
{
    const double a = (double)R + 1.0, b = (double)(N - R);
    const double ld = log(delta);
    const bool small = R < CP_SMALL_R && N - R > CP_SMALL_R;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
        double lpdf;
        double lF = small ? log_binom_cdf_small_warp(R, N, u, &lpdf, lane)
                          : log_binom_cdf_warp(a, b, u, &lpdf, lane);
        lF = __shfl_sync(0xffffffffu, lF, 0);   // keep the control flow warp-uniform
        lpdf = __shfl_sync(0xffffffffu, lpdf, 0);
        const double f = lF - ld;
        if (f == 0.0) break;
        const double r = exp(lpdf - lF);
        const double p1 = -r;
        const double p2 = -r * ((a - 1.0) / u - (b - 1.0) / (1.0 - u)) - r * r;
        const double den = 2.0 * p1 * p1 - f * p2;
        const double du = (den != 0.0) ? -2.0 * f * p1 / den : -f / p1;
        if (fabs(du) <= 4e-16 * u) break;
        if (f > 0.0) lo = u; else hi = u;
        double un = u + du;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        const double step = fabs(un - u);
        u = un;
        if (step <= 3e-6 * fmin(u, 1.0 - u) || hi - lo <= 4e-16 * hi) break;
    }
    return u;
}


// Device-side argument checks of tile i: a tile must meet some null hypothesis
// (null_mask != 0) and have half-widths h >= 0 (h = 0: a point); false and the
// error flag (reported by cse_sync as DEVICE_CHECK) otherwise.
template <int D>
__device__ bool tile_args_ok(const TileArgs& T, int64_t i, int32_t* err)
{
    bool ok = T.null_mask[i] != 0u;
#pragma unroll
    for (int a = 0; a < D; ++a) ok &= T.halfwidth[i * D + a] >= 0.0;   // false for NaN too
    if (!ok) atomicOr(err, CSE_ERR_BAD_K);
    return ok;
}

// Loads tile i's centre and half-widths; false (and the error flag) when an
// axis index is out of range or tile_args_ok fails.
template <int D>
__device__ bool load_tile(const TileArgs& T, int64_t i, double n_max, ArmGeom* G, int32_t* err)
{
    if (!tile_args_ok<D>(T, i, err)) return false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int v = T.center_idx[i * D + a];
        if (v < 0 || v >= T.n_axis[a]) {
            atomicOr(err, CSE_ERR_BAD_K);
            return false;
        }
        arm_init(G[a], T.axis[a][v], T.halfwidth[i * D + a], n_max);
    }
    return true;
}

// The per-arm softplus terms of a tile (sp(th), sp(th + h) - sp(th),
// sp(th - h) - sp(th)), 3 doubles per arm, as k_alpha_prime computed them:
// k_bounds of the same step reads them instead of recomputing (same values).
template <int D>
__device__ void store_geom(const ArmGeom* G, int64_t i, double* __restrict__ geom)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        geom[(i * D + a) * 3 + 0] = G[a].sp0;
        geom[(i * D + a) * 3 + 1] = G[a].d1p;
        geom[(i * D + a) * 3 + 2] = G[a].d1m;
    }
}

template <int D>
__device__ bool load_tile_geom(const TileArgs& T, int64_t i, double n_max, ArmGeom* G, int32_t* err,
                               const double* __restrict__ geom)
{
    if (!tile_args_ok<D>(T, i, err)) return false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int v = T.center_idx[i * D + a];
        if (v < 0 || v >= T.n_axis[a]) {
            atomicOr(err, CSE_ERR_BAD_K);
            return false;
        }
        G[a].th = T.axis[a][v];
        G[a].h = T.halfwidth[i * D + a];
        G[a].n = n_max;
        G[a].sp0 = geom[(i * D + a) * 3 + 0];
        G[a].d1p = geom[(i * D + a) * 3 + 1];
        G[a].d1m = geom[(i * D + a) * 3 + 2];
    }
    return true;
}

// Clopper-Pearson depends on a tile only through (R, K): every distinct pair is
// solved once.  k_cp_mark inserts each tile's key (K << 32 | R) into an
// open-addressing hash table (linear probing, at most `cap` probes, no waiting)
// and records its slot; k_cp_solve solves each occupied slot; k_bounds reads it.
constexpr unsigned long long kEmptyKey = kCpEmptyKey;

__global__ void k_cp_mark(int64_t n_tiles, const int64_t* __restrict__ R, const int32_t* __restrict__ K,
                          unsigned long long* __restrict__ keys, uint32_t cap, int32_t* __restrict__ slot,
                          uint32_t* __restrict__ list, int32_t* __restrict__ n_keys, bool lower)
{
    pdl_entry();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tiles) return;
    // Upper bound: the solve for R at delta.  Lower bound (see k_bounds): for
    // R > K/2 the upper solve for the K - R failures at delta, else the solve
    // for R - 1 at 1 - delta, tagged by the key's top bit; R = 0 needs none.
    int64_t Rk = R[i];
    unsigned long long tag = 0ull;
    if (lower) {
        if (2 * R[i] > (int64_t)K[i]) {
            Rk = (int64_t)K[i] - R[i];
        } else {
            Rk = R[i] - 1;
            tag = 1ull << 63;
        }
        if (Rk < 0) {
            slot[i] = -1;
            return;
        }
    }
    const unsigned long long key = tag | ((unsigned long long)(uint32_t)K[i] << 32) | (uint32_t)Rk;
    slot[i] = cp_memo_insert(key, keys, cap, list, n_keys);
}

// Distinct (K, R) keys 0 .. n_warp-1 take one warp each (the latency of one
// key is the solve's critical path when keys are few): 4 rounds of 32 FP32
// evaluations (one per lane) narrow the root to ~1e-6 relative, then the warp
// finishes it in FP64.  Key w goes to block w % warp_blocks, so keys spread
// over the SMs before they share one.  Keys beyond n_warp (many distinct keys:
// throughput matters) take one thread each in the remaining blocks, which run
// beside the warp blocks.  (16 warps a block with one key each took the
// two-arm 256^2 solve from 66 to 56 us, but at 128 registers a block then
// fills an SM, the thread blocks wait for the warp blocks, and the 2^18 batch
// and the basket lost 0.45 and 0.52 ms.)
constexpr int CP_WARPS_PER_BLOCK = 4;
constexpr int CP_KEYS_PER_WARP = 2;

__global__ void __launch_bounds__(32 * CP_WARPS_PER_BLOCK) k_cp_solve(unsigned long long* __restrict__ keys,
                                                  const uint32_t* __restrict__ list,
                                                  const int32_t* __restrict__ n_keys, double delta0,
                                                  double delta1, double* __restrict__ u0s, int warp_blocks)
{
    pdl_entry();
    const int n = *n_keys;
    const int n_warp = min(n, warp_blocks * CP_WARPS_PER_BLOCK * CP_KEYS_PER_WARP);
    if ((int)blockIdx.x < warp_blocks) {
        const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
        for (int w = blockIdx.x + warp_blocks * wib; w < n_warp; w += warp_blocks * CP_WARPS_PER_BLOCK) {
            const uint32_t h = list[w];
            const unsigned long long key = keys[h];
            const int64_t R = (int64_t)(uint32_t)key, N = (int64_t)((key >> 32) & 0x7FFFFFFFull);
            const double delta = (key >> 63) ? delta1 : delta0;
            if (R >= N || R <= 0) {
                if (lane == 0) {
                    u0s[h] = R >= N ? 1.0 : -expm1(log(delta) / (double)N);
                    keys[h] = kEmptyKey;   // the table is empty again for the next call
                }
                continue;
            }
            const float ldf = logf((float)delta);
            float lo, hi;
            cp_interval(R, N, &lo, &hi);
            for (int round = 0; round < 4; ++round) {
                float uj;
                cp_round_points(lo, hi, lane, &uj);
                const float f = cp_f32(R, N, uj, ldf, nullptr);
                const unsigned below = __ballot_sync(0xffffffffu, !(f > 0.0f));   // root at or left of uj
                if (below == 0u) {
                    lo = __shfl_sync(0xffffffffu, uj, 31);
                } else {
                    const int jf = __ffs(below) - 1;
                    const float uj_hi = __shfl_sync(0xffffffffu, uj, jf);
                    const float uj_lo = __shfl_sync(0xffffffffu, uj, jf > 0 ? jf - 1 : 0);
                    hi = uj_hi;
                    if (jf > 0) lo = uj_lo;
                }
            }
            // The FP64 stage is safeguarded on [0, 1]: an FP32 bracket that missed
            // the FP64 root only costs it extra steps.
            const double u = cp_finish_warp(R, N, delta, 0.5 * ((double)lo + (double)hi), lane);
            if (lane == 0) {
                u0s[h] = u;
                keys[h] = kEmptyKey;
            }
        }
        return;
    }
    const int stride = (gridDim.x - warp_blocks) * blockDim.x;
    for (int t = n_warp + (blockIdx.x - warp_blocks) * blockDim.x + threadIdx.x; t < n; t += stride) {
        const uint32_t h = list[t];
        const unsigned long long key = keys[h];
        const int64_t R = (int64_t)(uint32_t)key, N = (int64_t)((key >> 32) & 0x7FFFFFFFull);
        u0s[h] = cp_upper(R, N, (key >> 63) ? delta1 : delta0);
        keys[h] = kEmptyKey;
    }
}

// Upper: u0 = Clopper-Pearson upper bound of R / K, bound = optimised tile
// Tilt-Bound.  LOWER (Rem. extension-lower): u0 = lower Clopper-Pearson bound
// l (P(Binom(K, l) >= R) = delta), bound = 1 - U_tile(1 - l) = -expm1(log U_tile).
// 1 - l enters as log(1 - l): for R <= K/2 l is the upper solve for R - 1 at
// 1 - delta and log(1 - l) = log1p(-l); for R > K/2 (l near 1) 1 - l is the
// upper solve for the K - R failures at delta (binomial symmetry), taken
// directly so that its digits are not lost to the subtraction.
template <int D, bool PLAIN, bool LOWER>
__global__ void __launch_bounds__(128) k_bounds(TileArgs T, int32_t n_max, const int64_t* __restrict__ R,
                                                double delta, double* __restrict__ u0,
                                                double* __restrict__ bound, double* __restrict__ qstar,
                                                int32_t* __restrict__ err, const int32_t* __restrict__ slot,
                                                const double* __restrict__ u0s, const double* __restrict__ geom,
                                                int32_t* __restrict__ nkeys_reset)
{
    pdl_entry();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n_tiles) return;
    // k_cp_solve has read the key count (it ran before this kernel): zero it for the next call
    if (i == 0 && nkeys_reset) *nkeys_reset = 0;
    ArmGeom G[D];
    const bool ok = geom ? load_tile_geom<D>(T, i, (double)n_max, G, err, geom)
                         : load_tile<D>(T, i, (double)n_max, G, err);
    if (!ok) {
        if (u0) u0[i] = NAN;
        if (bound) bound[i] = NAN;
        if (qstar) qstar[i] = NAN;
        return;
    }
    double q;
    if (LOWER) {
        const int64_t Ri = R[i], Ki = T.K[i];
        const bool memo = !PLAIN && slot && slot[i] >= 0;
        double l, la;
        if (2 * Ri > Ki) {
            const double ap = PLAIN ? cp_upper_plain(Ki - Ri, Ki, delta)
                                    : memo ? u0s[slot[i]] : cp_upper(Ki - Ri, Ki, delta);
            l = 1.0 - ap;
            la = log(ap);
        } else if (Ri <= 0) {
            l = 0.0;
            la = 0.0;
        } else {
            l = PLAIN ? cp_upper_plain(Ri - 1, Ki, 1.0 - delta)
                      : memo ? u0s[slot[i]] : cp_upper(Ri - 1, Ki, 1.0 - delta);
            la = log1p(-l);
        }
        const double lb = tilt_bound_log_la<D, PLAIN>(G, la, &q);
        if (u0) u0[i] = l;
        if (bound) bound[i] = (lb >= 0.0) ? 0.0 : -expm1(lb);
        if (qstar) qstar[i] = q;
        return;
    }
    double u;
    if (PLAIN) u = cp_upper_plain(R[i], T.K[i], delta);
    else if (slot && slot[i] >= 0) u = u0s[slot[i]];
    else u = cp_upper(R[i], T.K[i], delta);
    const double lb = tilt_bound_log<D, PLAIN>(G, u, &q);
    if (u0) u0[i] = u;
    if (bound) bound[i] = exp(lb);
    if (qstar) qstar[i] = q;
}

template <int D, bool PLAIN>
__global__ void __launch_bounds__(128) k_alpha_prime(TileArgs T, int32_t n_max, double alpha,
                                                     double* __restrict__ aprime, int32_t* __restrict__ ksel,
                                                     int32_t* __restrict__ err, double* __restrict__ geom)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n_tiles) return;
    ArmGeom G[D];
    if (!load_tile<D>(T, i, (double)n_max, G, err)) {
        if (aprime) aprime[i] = NAN;
        if (ksel) ksel[i] = 0;
        return;
    }
    if (geom) store_geom<D>(G, i, geom);
    double q;
    const double ap = exp(alpha_prime_log<D, PLAIN>(G, alpha, &q));
    if (aprime) aprime[i] = ap;
    const int32_t K = T.K[i];
    double kf = floor(((double)K + 1.0) * ap);
    if (kf > (double)K) kf = (double)K;
    if (ksel) ksel[i] = (int32_t)kf;
}


// min over v[0..n): each block folds its stretch on integer keys (ALU, not the
// FP64 pipe), one atomicMin per block into *key (set to all ones before the
// launch), and the last block to finish (a ticket counter, no waiting) writes
// the decoded minimum and resets the ticket.
__global__ void __launch_bounds__(256) k_min(const double* __restrict__ v, int64_t n, double* __restrict__ out,
                                             unsigned long long* __restrict__ key, unsigned int* __restrict__ ticket)
{
    pdl_entry();
    __shared__ unsigned long long red[8];
    __shared__ bool last;
    unsigned long long m = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = min(m, order_key(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = min(m, red[w]);
        atomicMin(key, m);
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long k = atomicAdd(key, 0ull);
        *out = (k == ~0ull) ? INFINITY : order_unkey(k);
        *key = ~0ull;   // reset for the next launch
        *ticket = 0u;
    }
}

__global__ void k_backward(int64_t n, int32_t d, const double* __restrict__ g, const double* __restrict__ score,
                           const int32_t* __restrict__ K, double* __restrict__ out)
{
    pdl_entry();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * d) return;
    const int64_t i = j / d;
    out[j] = g[i] * score[j] / (double)K[i];
}

}  // namespace

template <int D>
void launch_bounds_d(cse_ctx* c, unsigned blocks, const TileArgs& T, const int64_t* R, double delta, bool lower,
                     double* u0, double* bound, double* qstar, const int32_t* slot, const double* geom,
                     cudaStream_t s)
{
    const int nm = c->D.n_max;
    if (c->plain) {
        if (lower)
            cse_launch(c->pdl, k_bounds<D, true, true>, dim3(blocks), dim3(128), 0, s, T, nm, R, delta, u0, bound, qstar, c->err, nullptr, nullptr,
                                                           nullptr, nullptr);
        else
            cse_launch(c->pdl, k_bounds<D, true, false>, dim3(blocks), dim3(128), 0, s, T, nm, R, delta, u0, bound, qstar, c->err, nullptr,
                                                            nullptr, nullptr, nullptr);
    } else {
        // one thread a tile, 64-thread blocks: the tiles spread over more SMs
        // than in blocks of 128 (two-arm 256^2: 66 -> 62 us, refined sample
        // 272 -> 243 us)
        int32_t* nk = slot ? c->cp_nkeys : nullptr;
        const unsigned b64 = (unsigned)((T.n_tiles + 63) / 64);
        if (lower)
            cse_launch(c->pdl, k_bounds<D, false, true>, dim3(b64), dim3(64), 0, s, T, nm, R, delta, u0, bound, qstar, c->err, slot,
                                                            c->cp_val, geom, nk);
        else
            cse_launch(c->pdl, k_bounds<D, false, false>, dim3(b64), dim3(64), 0, s, T, nm, R, delta, u0, bound, qstar, c->err, slot,
                                                             c->cp_val, geom, nk);
    }
}

template <int D>
void launch_alpha_d(cse_ctx* c, unsigned blocks, const TileArgs& T, double alpha, double* ap, int32_t* ksel,
                    double* geom, cudaStream_t s)
{
    if (c->plain)
        k_alpha_prime<D, true><<<blocks, 128, 0, s>>>(T, c->D.n_max, alpha, ap, ksel, c->err, nullptr);
    else
        k_alpha_prime<D, false><<<blocks, 128, 0, s>>>(T, c->D.n_max, alpha, ap, ksel, c->err, geom);
}

int cse_launch_bounds(cse_ctx* c, const TileArgs& T, const int64_t* R, double delta, bool lower, double* u0,
                      double* bound, double* qstar, cudaStream_t s, const double* geom, bool marked)
{
    const unsigned blocks = (unsigned)((T.n_tiles + 127) / 128);
    const int32_t* slot = nullptr;
    if (!c->plain && c->cp_cap >= 2 * (uint64_t)T.n_tiles) {
        // one Clopper-Pearson solve per distinct (R, K)
        // the key table is empty and the key count zero on entry: k_cp_solve empties
        // the slots it solves and k_bounds zeroes the count (both set at allocation)
        cse_prof_begin(c, KID_CP, s);
        if (!(marked && !lower)) {
            cse_launch(c->pdl, k_cp_mark, dim3(blocks), dim3(128), 0, s, T.n_tiles, R, T.K, c->cp_key,
                       (uint32_t)c->cp_cap, c->cp_slot, c->cp_list, c->cp_nkeys, lower);
            c->launches += 1;
        }
        const int64_t warp_keys = (int64_t)c->num_sms * CP_WARPS_PER_BLOCK * CP_KEYS_PER_WARP;
        constexpr int cp_threads = 32 * CP_WARPS_PER_BLOCK;
        const int64_t thread_blocks = std::max<int64_t>(0, (T.n_tiles - warp_keys + cp_threads - 1) / cp_threads);
        cse_launch(c->pdl, k_cp_solve, dim3((unsigned)(c->num_sms + thread_blocks)), dim3(cp_threads), 0,
                   s, c->cp_key, c->cp_list, c->cp_nkeys, delta, 1.0 - delta, c->cp_val, c->num_sms);
        cse_prof_end(c, s);
        c->launches += 1;
        slot = c->cp_slot;
    }
    cse_prof_begin(c, KID_BOUNDS, s);
    switch (T.d) {
    case 1: launch_bounds_d<1>(c, blocks, T, R, delta, lower, u0, bound, qstar, slot, geom, s); break;
    case 2: launch_bounds_d<2>(c, blocks, T, R, delta, lower, u0, bound, qstar, slot, geom, s); break;
    case 4: launch_bounds_d<4>(c, blocks, T, R, delta, lower, u0, bound, qstar, slot, geom, s); break;
    default: return CSE_UNSUPPORTED_DESIGN;
    }
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

// k_alpha_prime runs beside the table kernels (second stream) and uses no
// shared memory.  Left to itself its SMs take a small shared-memory carveout,
// and a table kernel's blocks (16 KB of shared memory each) then wait on every
// SM until the alpha' blocks there have finished, as an SM changes its
// carveout only when idle.  Asking for the largest carveout lets both run.
int cse_bound_set_attrs()
{
    const int pref = cudaSharedmemCarveoutMaxShared;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<1, false>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<2, false>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<4, false>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<1, true>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<2, true>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_alpha_prime<4, true>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    return e == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_alpha_prime(cse_ctx* c, const TileArgs& T, double alpha, double* aprime_out,
                           int32_t* ksel, cudaStream_t s, double* geom)
{
    const unsigned blocks = (unsigned)((T.n_tiles + 127) / 128);
    cse_prof_begin(c, KID_ALPHA_PRIME, s);
    switch (T.d) {
    case 1: launch_alpha_d<1>(c, blocks, T, alpha, aprime_out, ksel, geom, s); break;
    case 2: launch_alpha_d<2>(c, blocks, T, alpha, aprime_out, ksel, geom, s); break;
    case 4: launch_alpha_d<4>(c, blocks, T, alpha, aprime_out, ksel, geom, s); break;
    default: return CSE_UNSUPPORTED_DESIGN;
    }
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_min(cse_ctx* c, const double* lam_tile, int64_t n, double* out, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 2 * (int64_t)c->num_sms) blocks = 2 * (int64_t)c->num_sms;
    if (blocks < 1) blocks = 1;
    // min_key is all ones and the ticket zero on entry (set at creation, restored by the last block)
    cse_prof_begin(c, KID_MIN, s);
    cse_launch(c->pdl, k_min, dim3((unsigned)blocks), dim3(256), 0, s, lam_tile, n, out, c->min_key, c->min_ticket);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_backward(int64_t n, int32_t d, const double* g, const double* score, const int32_t* K,
                        double* out, cudaStream_t s)
{
    const int64_t tot = n * d;
    if (tot == 0) return CSE_OK;
    cse_launch(true, k_backward, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, s, n, d, g, score, K, out);
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

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

#include "cse_internal.cuh"

namespace {

constexpr double SMAX = 40.0;   // search range s = log q in [0, 40]
constexpr int BISECT_IT = 64;

struct ArmGeom {
    double th, h, n, sp0, d1p, d1m;   // d1p/d1m = sp(th +/- h) - sp(th)
};

__device__ __forceinline__ double softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

__device__ __forceinline__ void arm_init(ArmGeom& g, double th, double h, double n)
{
    g.th = th;
    g.h = h;
    g.n = n;
    g.sp0 = softplus(th);
    g.d1p = softplus(th + h) - g.sp0;
    g.d1m = softplus(th - h) - g.sp0;
}

// Phi(q) = sum_a max_{s=+-1} phi_a(q, s h_a) and its q-derivative along the
// maximising branch (the larger derivative on a tie: the right derivative).
__device__ void tilt_phi(const ArmGeom* G, int d, double q, double* Phi, double* dPhi)
{
    double P = 0.0, dP = 0.0;
    const double iq = 1.0 / q;
    for (int a = 0; a < d; ++a) {
        double best = -INFINITY, bestd = 0.0;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const double v = sg ? -G[a].h : G[a].h;
            const double x = G[a].th + q * v;
            const double e = exp(-fabs(x));
            const double sp = fmax(x, 0.0) + log1p(e) - G[a].sp0;
            const double sig = ((x >= 0.0) ? 1.0 : e) / (1.0 + e);
            const double phi = G[a].n * (sp * iq - (sg ? G[a].d1m : G[a].d1p));
            const double dphi = G[a].n * (q * v * sig - sp) * iq * iq;
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

// lim_{q->inf} Phi(q) = sum_a max(n h_a - n d1p, -n d1m)
__device__ double tilt_phi_inf(const ArmGeom* G, int d)
{
    double P = 0.0;
    for (int a = 0; a < d; ++a) P += G[a].n * fmax(G[a].h - G[a].d1p, -G[a].d1m);
    return P;
}

// inf_q max_v U(theta0, v, q, a); returns log bound, *qstar.
__device__ double tilt_bound_log(const ArmGeom* G, int d, double a, double* qstar)
{
    if (a >= 1.0) {
        *qstar = 1.0;
        return 0.0;
    }
    if (!(a > 0.0)) {
        *qstar = INFINITY;
        return -INFINITY;
    }
    const double la = log(a);
    double lo = 0.0, hi = SMAX;
    for (int it = 0; it < BISECT_IT; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double q = exp(mid);
        double P, dP;
        tilt_phi(G, d, q, &P, &dP);
        const double g1 = la / (q * q) + dP;
        if (g1 < 0.0) lo = mid; else hi = mid;
    }
    const double s = 0.5 * (lo + hi);
    double q = exp(s);
    double P, dP;
    tilt_phi(G, d, q, &P, &dP);
    double val = (1.0 - 1.0 / q) * la + P;
    if (s > SMAX - 1e-6) {
        const double vinf = la + tilt_phi_inf(G, d);
        if (vinf <= val) {
            *qstar = INFINITY;
            return vinf;
        }
    }
    *qstar = q;
    return val;
}

// sup_q min_v U^-1(theta0, v, q, alpha); returns log alpha', *qstar.
__device__ double alpha_prime_log(const ArmGeom* G, int d, double alpha, double* qstar)
{
    const double lal = log(alpha);
    double lo = 0.0, hi = SMAX;
    for (int it = 0; it < BISECT_IT; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double q = exp(mid);
        double P, dP;
        tilt_phi(G, d, q, &P, &dP);
        // sign of dM/dq for M = q/(q-1) (log alpha - Phi)
        const double sgn = -lal + P - q * (q - 1.0) * dP;
        if (sgn > 0.0) lo = mid; else hi = mid;
    }
    const double s = 0.5 * (lo + hi);
    const double q = exp(s);
    double P, dP;
    tilt_phi(G, d, q, &P, &dP);
    double val = q / (q - 1.0) * (lal - P);
    if (s > SMAX - 1e-6) {
        const double vinf = lal - tilt_phi_inf(G, d);
        if (vinf >= val) {
            *qstar = INFINITY;
            return vinf;
        }
    }
    *qstar = q;
    return val;
}

// ---------------------------------------------------------------------------
// Clopper-Pearson (Eq. clopper-pearson:def): u with P(Binom(N, u) <= R) = delta,
// i.e. I_{1-u}(N - R, R + 1) = delta, by safeguarded Newton in log space on the
// regularised incomplete beta function, evaluated by its continued fraction
// (modified Lentz) with a Stirling-series prefactor for large parameters.
// ---------------------------------------------------------------------------

// Stirling-series remainder lgamma(z) - [(z - 1/2) log z - z + log(2 pi)/2], z >= 10.
__device__ __forceinline__ double stirling_rem(double z)
{
    const double r = 1.0 / z, r2 = r * r;
    return r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0 - r2 * (1.0 / 1680.0 - r2 / 1188.0))));
}

// log(x^a y^b / B(a, b)) with lx = log x, ly = log y (y = 1 - x) and
// e = x (a + b) - a supplied accurately by the caller.
__device__ double log_bpre(double a, double b, double lx, double ly, double e)
{
    const double L2PI = 1.8378770664093454836;
    if (a >= 10.0 && b >= 10.0) {
        return a * log1p(e / a) + b * log1p(-e / b) + 0.5 * log(a * b / (a + b)) - 0.5 * L2PI
               - (stirling_rem(a) + stirling_rem(b) - stirling_rem(a + b));
    }
    if (b >= 10.0) {   // small a: lgamma(a+b) - lgamma(b) by the Stirling difference
        return a * lx + b * ly - lgamma(a) + a * log(a + b) + (b - 0.5) * log1p(a / b) - a
               + stirling_rem(a + b) - stirling_rem(b);
    }
    if (a >= 10.0) {
        return a * lx + b * ly - lgamma(b) + b * log(a + b) + (a - 0.5) * log1p(b / a) - b
               + stirling_rem(a + b) - stirling_rem(a);
    }
    return a * lx + b * ly - lgamma(a) - lgamma(b) + lgamma(a + b);
}

// Continued fraction of I_x(a, b) (modified Lentz): I = x^a y^b / (a B) * cf.
__device__ double beta_cf(double a, double b, double x)
{
    const double TINY = 1e-300;
    const double qab = a + b, qap = a + 1.0, qam = a - 1.0;
    double c = 1.0, dd = 1.0 - qab * x / qap;
    if (fabs(dd) < TINY) dd = TINY;
    dd = 1.0 / dd;
    double h = dd;
    for (int m = 1; m <= 4000; ++m) {
        const double m2 = 2.0 * m;
        double aa = m * (b - m) * x / ((qam + m2) * (a + m2));
        dd = 1.0 + aa * dd;
        if (fabs(dd) < TINY) dd = TINY;
        c = 1.0 + aa / c;
        if (fabs(c) < TINY) c = TINY;
        dd = 1.0 / dd;
        h *= dd * c;
        aa = -(a + m) * (qab + m) * x / ((a + m2) * (qap + m2));
        dd = 1.0 + aa * dd;
        if (fabs(dd) < TINY) dd = TINY;
        c = 1.0 + aa / c;
        if (fabs(c) < TINY) c = TINY;
        dd = 1.0 / dd;
        const double del = dd * c;
        h *= del;
        if (fabs(del - 1.0) <= 2.2e-16) break;
    }
    return h;
}

// log P(Binom(N, u) <= R) = log I_{1-u}(b, a), a = R + 1, b = N - R.
__device__ double log_binom_cdf(double a, double b, double u)
{
    const double lu = log(u), l1u = log1p(-u);
    const double e = fma(u, a + b, -a);   // u (a+b) - a
    if (u >= (a + 1.0) / (a + b + 2.0)) {
        // I_{1-u}(b, a) directly: x' = 1 - u, e' = (1-u)(a+b) - b = -e
        const double lp = log_bpre(b, a, l1u, lu, -e);
        return lp + log(beta_cf(b, a, 1.0 - u)) - log(b);
    }
    const double lp = log_bpre(a, b, lu, l1u, e);
    const double I = exp(lp) * beta_cf(a, b, u) / a;   // I_u(a, b)
    return log1p(-I);
}

__device__ double cp_upper(int64_t R, int64_t N, double delta)
{
    if (R >= N) return 1.0;
    if (R <= 0) return -expm1(log(delta) / (double)N);
    const double a = (double)R + 1.0, b = (double)(N - R);
    const double ld = log(delta);
    const double mean = a / (a + b);
    const double sd = sqrt(a * b / ((a + b) * (a + b) * (a + b + 1.0)));
    double lo = 0.0, hi = 1.0;
    double u = fmin(mean + 2.5 * sd, 0.5 * (mean + 1.0));
    for (int it = 0; it < 200; ++it) {
        const double lF = log_binom_cdf(a, b, u);
        const double f = lF - ld;
        if (f > 0.0) lo = u; else hi = u;
        const double lu = log(u), l1u = log1p(-u);
        const double lpdf = log_bpre(a, b, lu, l1u, fma(u, a + b, -a)) - lu - l1u;
        const double dlF = -exp(lpdf - lF);
        double un = u - f / dlF;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        if (fabs(un - u) <= 2e-16 * u || hi - lo <= 2e-16 * hi) {
            u = un;
            break;
        }
        u = un;
    }
    return u;
}

// Loads tile i's centre and half-widths; false (and the error flag) when an
// axis index is out of range.
__device__ bool load_tile(const TileArgs& T, int64_t i, double n_max, ArmGeom* G, int32_t* err)
{
    for (int a = 0; a < T.d; ++a) {
        const int v = T.center_idx[i * T.d + a];
        if (v < 0 || v >= T.n_axis[a]) {
            atomicOr(err, CSE_ERR_BAD_K);
            return false;
        }
        arm_init(G[a], T.axis[a][v], T.halfwidth[i * T.d + a], n_max);
    }
    return true;
}

__global__ void __launch_bounds__(128) k_bounds(TileArgs T, int32_t n_max, const int64_t* __restrict__ R,
                                                double delta, double* __restrict__ u0,
                                                double* __restrict__ bound, double* __restrict__ qstar,
                                                int32_t* __restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n_tiles) return;
    const int d = T.d;
    ArmGeom G[CSE_MAX_ARMS];
    if (!load_tile(T, i, (double)n_max, G, err)) {
        if (u0) u0[i] = NAN;
        if (bound) bound[i] = NAN;
        if (qstar) qstar[i] = NAN;
        return;
    }
    const double u = cp_upper(R[i], T.K[i], delta);
    double q;
    const double lb = tilt_bound_log(G, d, u, &q);
    if (u0) u0[i] = u;
    if (bound) bound[i] = exp(lb);
    if (qstar) qstar[i] = q;
}

__global__ void __launch_bounds__(128) k_alpha_prime(TileArgs T, int32_t n_max, double alpha,
                                                     double* __restrict__ aprime, int32_t* __restrict__ ksel,
                                                     int32_t* __restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n_tiles) return;
    const int d = T.d;
    ArmGeom G[CSE_MAX_ARMS];
    if (!load_tile(T, i, (double)n_max, G, err)) {
        if (aprime) aprime[i] = NAN;
        if (ksel) ksel[i] = 0;
        return;
    }
    double q;
    const double ap = exp(alpha_prime_log(G, d, alpha, &q));
    if (aprime) aprime[i] = ap;
    const int32_t K = T.K[i];
    double kf = floor(((double)K + 1.0) * ap);
    if (kf > (double)K) kf = (double)K;
    if (ksel) ksel[i] = (int32_t)kf;
}

// min over tiles, one block of 1024 threads (n is at most a few million)
__global__ void __launch_bounds__(1024) k_min(const double* __restrict__ v, int64_t n, double* __restrict__ out)
{
    __shared__ double red[32];
    double m = INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

__global__ void k_backward(int64_t n, int32_t d, const double* __restrict__ g, const double* __restrict__ score,
                           const int32_t* __restrict__ K, double* __restrict__ out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * d) return;
    const int64_t i = j / d;
    out[j] = g[i] * score[j] / (double)K[i];
}

}  // namespace

int cse_launch_bounds(cse_ctx* c, const TileArgs& T, const int64_t* R, double delta, double* u0,
                      double* bound, double* qstar, cudaStream_t s)
{
    const int64_t blocks = (T.n_tiles + 127) / 128;
    cse_prof_begin(c, KID_BOUNDS, s);
    k_bounds<<<(unsigned)blocks, 128, 0, s>>>(T, c->D.n_max, R, delta, u0, bound, qstar, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_alpha_prime(cse_ctx* c, const TileArgs& T, double alpha, double* aprime_out,
                           int32_t* ksel, cudaStream_t s)
{
    const int64_t blocks = (T.n_tiles + 127) / 128;
    cse_prof_begin(c, KID_ALPHA_PRIME, s);
    k_alpha_prime<<<(unsigned)blocks, 128, 0, s>>>(T, c->D.n_max, alpha, aprime_out, ksel, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_min(cse_ctx* c, const double* lam_tile, int64_t n, double* out, cudaStream_t s)
{
    cse_prof_begin(c, KID_MIN, s);
    k_min<<<1, 1024, 0, s>>>(lam_tile, n, out);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_backward(int64_t n, int32_t d, const double* g, const double* score, const int32_t* K,
                        double* out, cudaStream_t s)
{
    const int64_t tot = n * d;
    if (tot == 0) return CSE_OK;
    k_backward<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, d, g, score, K, out);
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

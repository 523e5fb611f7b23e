// sim_bayes4.cu -- the four-arm Bayesian selection design (control + 3
// treatments, interim analyses after look_n[0] and look_n[1] patients per arm,
// final analysis after look_n[2]) with the hierarchical model of Sec. 10.1:
//   theta_i ~ N(mu, s2), mu ~ N(-1.34, 100), s2 ~ InvGamma(0.0005, 0.000005),
// each arm's likelihood replaced by the normal approximation of its empirical
// logit, s2 integrated on 16 log-spaced nodes in [1e-6, 1e3] (trapezoid in
// log s2, weights normalised by log-sum-exp), mu and theta integrated exactly.
// Interim: drop treatment i when P(theta_i > theta_0 | data) < drop (its data
// stay in the model, frozen).  Final: S = min over active true-null arms of
// 1 - P_i; reject iff S < lambda.  The posterior runs in FP32.
//
// The design depends on a simulated trial only through its success counts, so
// the posterior is tabulated once per context over every reachable count state
// (interim drop decisions and final-look probabilities); a simulation then costs
// count reads and a few table reads.  Treatments are exchangeable in the model,
// so the final-look table holds, per control count and sorted triple of
// treatment codes, the three P(theta_self > theta_0) side by side (one float4:
// one 16-byte read per trial), each evaluated with the arms in the canonical
// order (control, self, the other two ascending).  A direct mode evaluates the
// same FP32 posterior function per simulation instead of reading tables.
#include <cuda_runtime.h>
#include <math.h>

#include "cse_internal.cuh"

namespace {

constexpr int NODES = kBayesNodes;   // quadrature nodes of s2 (node_const)
constexpr int BT = 256;          // threads of the simulation kernel
constexpr int BWARP = BT / 32;

// P(theta_i > theta_0 | data) for i = 1..3 in FP32.  Not inlined, so every caller
// runs the same instruction sequence (identical results for identical inputs).
__device__ __noinline__ void posterior4_f32(const int* x, const int* n, const NodeConst& C, float* P)
{
    const float MU0 = -1.34f, TAU2 = 100.0f;
    float th[4], s2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float xs = (float)x[i] + 0.5f, fs = (float)(n[i] - x[i]) + 0.5f;
        th[i] = logf(xs / fs);
        s2[i] = 1.0f / xs + 1.0f / fs;
    }
    float lw[NODES], pj[NODES][3];
    float mx = -INFINITY;
#pragma unroll 4
    for (int j = 0; j < NODES; ++j) {
        const float sg = C.sig2[j];
        float W = 0.f, Sr = 0.f, Srr = 0.f, Sth = 0.f, prod = 1.f;
        float w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float den = sg + s2[i];
            w[i] = 1.0f / den;
            const float r = th[i] - MU0;
            W += w[i];
            Sr += w[i] * r;
            Srr += w[i] * r * r;
            Sth += w[i] * th[i];
            prod *= den;
        }
        const float prec = 1.0f / TAU2 + W;
        const float quad = Srr - Sr * Sr / prec;
        const float logdet = logf(prod * (1.0f + TAU2 * W));
        lw[j] = C.lprior[j] - 0.5f * logdet - 0.5f * quad;
        mx = fmaxf(mx, lw[j]);
        const float mmu = (MU0 / TAU2 + Sth) / prec;
        const float vmu = 1.0f / prec;
        float c[4], v[4], e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            c[i] = s2[i] * w[i];
            v[i] = s2[i] * sg * w[i];
            e[i] = (1.0f - c[i]) * th[i] + c[i] * mmu;
        }
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            const float md = e[i] - e[0];
            const float dc = c[i] - c[0];
            const float vd = v[i] + v[0] + dc * dc * vmu;
            pj[j][i - 1] = normcdff(md * rsqrtf(vd));
        }
    }
    float Z = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
        const float wj = expf(lw[j] - mx);
        Z += wj;
        a0 += wj * pj[j][0];
        a1 += wj * pj[j][1];
        a2 += wj * pj[j][2];
    }
    P[0] = a0 / Z;
    P[1] = a1 / Z;
    P[2] = a2 / Z;
}

// Treatment-state codes: at the second analysis, code < n1+1 is "dropped at the
// first analysis with x successes of n1", else "active with x = code-(n1+1) of
// n2"; at the final analysis codes < n1+1 and < n1+1+n2+1 are dropped at the
// first / second analysis, the rest active with x = code-(n1+1)-(n2+1) of n3.
struct Looks {
    int n1, n2, n3, S2, S3, NP;   // NP = S3 (S3 + 1) / 2 unordered pairs
    int NT;                       // S3 (S3 + 1) (S3 + 2) / 6 sorted triples
};

// Position of the sorted triple a <= b <= c among all sorted triples of codes
// (combinatorial number system).
__device__ __forceinline__ int triple_index(int a, int b, int c)
{
    return c * (c + 1) * (c + 2) / 6 + b * (b + 1) / 2 + a;
}

__device__ __forceinline__ void decode3(const Looks& L, int code, int* x, int* n)
{
    if (code <= L.n1) {
        *x = code;
        *n = L.n1;
    } else if (code <= L.n1 + 1 + L.n2) {
        *x = code - (L.n1 + 1);
        *n = L.n2;
    } else {
        *x = code - (L.n1 + 1) - (L.n2 + 1);
        *n = L.n3;
    }
}

__global__ void k_table_d1(uint8_t* __restrict__ D1, Looks L, float drop)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = L.n1 + 1;
    if (s >= m * m * m * m) return;
    const NodeConst C = node_const();
    int x[4] = {s / (m * m * m), (s / (m * m)) % m, (s / m) % m, s % m};
    int n[4] = {L.n1, L.n1, L.n1, L.n1};
    float P[3];
    posterior4_f32(x, n, C, P);
    D1[s] = (uint8_t)((P[0] < drop ? 1 : 0) | (P[1] < drop ? 2 : 0) | (P[2] < drop ? 4 : 0));
}

__global__ void k_table_d2(uint8_t* __restrict__ D2, Looks L, float drop)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int S2 = L.S2;
    if (s >= (L.n2 + 1) * S2 * S2 * S2) return;
    const NodeConst C = node_const();
    const int c = s / (S2 * S2 * S2);
    const int t[3] = {(s / (S2 * S2)) % S2, (s / S2) % S2, s % S2};
    int x[4], n[4];
    x[0] = c;
    n[0] = L.n2;
    for (int i = 0; i < 3; ++i) {
        if (t[i] <= L.n1) {
            x[i + 1] = t[i];
            n[i + 1] = L.n1;
        } else {
            x[i + 1] = t[i] - (L.n1 + 1);
            n[i + 1] = L.n2;
        }
    }
    float P[3];
    posterior4_f32(x, n, C, P);
    D2[s] = (uint8_t)((P[0] < drop ? 1 : 0) | (P[1] < drop ? 2 : 0) | (P[2] < drop ? 4 : 0));
}

// F4[c * NT + triple_index(A, B, Z)] = (P_A, P_B, P_Z, 0) for the sorted codes
// A <= B <= Z: P_A = P(theta_A > theta_0) with the arms ordered (control, A, B, Z),
// P_B with (control, B, A, Z), P_Z with (control, Z, A, B).
__global__ void k_table_f4(float4* __restrict__ F4, Looks L)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(L.n3 + 1) * L.NT;
    if (s >= tot) return;
    const NodeConst C = node_const();
    const int c = (int)(s / L.NT);
    const int r = (int)(s % L.NT);
    int z = (int)cbrtf(6.0f * (float)r);   // largest z with z (z + 1) (z + 2) / 6 <= r
    while (z > 0 && z * (z + 1) * (z + 2) / 6 > r) --z;
    while ((z + 1) * (z + 2) * (z + 3) / 6 <= r) ++z;
    const int r2 = r - z * (z + 1) * (z + 2) / 6;
    int b = (int)floorf((sqrtf(8.0f * r2 + 1.0f) - 1.0f) * 0.5f);   // largest b with b (b + 1) / 2 <= r2
    while (b > 0 && b * (b + 1) / 2 > r2) --b;
    while ((b + 1) * (b + 2) / 2 <= r2) ++b;
    const int a = r2 - b * (b + 1) / 2;
    const int self[3] = {a, b, z}, lo[3] = {b, a, a}, hi[3] = {z, z, b};
    float out[3];
    for (int k = 0; k < 3; ++k) {
        int x[4], n[4];
        x[0] = c;
        n[0] = L.n3;
        decode3(L, self[k], &x[1], &n[1]);
        decode3(L, lo[k], &x[2], &n[2]);
        decode3(L, hi[k], &x[3], &n[3]);
        float P[3];
        posterior4_f32(x, n, C, P);
        out[k] = P[0];
    }
    F4[s] = make_float4(out[0], out[1], out[2], 0.0f);
}

// P_self at the final analysis evaluated directly, with the canonical arm order.
__device__ __forceinline__ float final_p_direct(const Looks& L, const NodeConst& C, int c, int self, int o1, int o2)
{
    const int ta = min(o1, o2), tb = max(o1, o2);
    int x[4], n[4];
    x[0] = c;
    n[0] = L.n3;
    decode3(L, self, &x[1], &n[1]);
    decode3(L, ta, &x[2], &n[2]);
    decode3(L, tb, &x[3], &n[3]);
    float P[3];
    posterior4_f32(x, n, C, P);
    return P[0];
}

// Statistic S of one simulated trial from its cumulative counts xl[look][arm].
template <bool TABLES>
__device__ __forceinline__ float design_stat(const Looks& L, const uint8_t* __restrict__ D1,
                                             const uint8_t* __restrict__ D2, const float4* __restrict__ F4,
                                             const NodeConst& C, float drop, const int xl[3][4], uint32_t mask)
{
    // first analysis: every arm at n1
    int bits;
    if (TABLES) {
        const int m = L.n1 + 1;
        // D1 may live in shared memory: a generic load (not the global-only __ldg)
        bits = D1[((xl[0][0] * m + xl[0][1]) * m + xl[0][2]) * m + xl[0][3]];
    } else {
        int x[4] = {xl[0][0], xl[0][1], xl[0][2], xl[0][3]};
        int n[4] = {L.n1, L.n1, L.n1, L.n1};
        float P[3];
        posterior4_f32(x, n, C, P);
        bits = (P[0] < drop ? 1 : 0) | (P[1] < drop ? 2 : 0) | (P[2] < drop ? 4 : 0);
    }
    int drop1 = bits & 7;                       // dropped at the first analysis
    if (drop1 == 7) return INFINITY;
    int t2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        t2[i] = ((drop1 >> i) & 1) ? xl[0][i + 1] : (L.n1 + 1) + xl[1][i + 1];
    if (TABLES) {
        bits = __ldg(D2 + ((xl[1][0] * L.S2 + t2[0]) * L.S2 + t2[1]) * L.S2 + t2[2]);
    } else {
        int x[4], n[4];
        x[0] = xl[1][0];
        n[0] = L.n2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const bool dr = (drop1 >> i) & 1;
            x[i + 1] = dr ? xl[0][i + 1] : xl[1][i + 1];
            n[i + 1] = dr ? L.n1 : L.n2;
        }
        float P[3];
        posterior4_f32(x, n, C, P);
        bits = (P[0] < drop ? 1 : 0) | (P[1] < drop ? 2 : 0) | (P[2] < drop ? 4 : 0);
    }
    const int drop2 = bits & 7 & ~drop1;        // dropped at the second analysis
    if ((drop1 | drop2) == 7) return INFINITY;
    int t3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if ((drop1 >> i) & 1) t3[i] = xl[0][i + 1];
        else if ((drop2 >> i) & 1) t3[i] = (L.n1 + 1) + xl[1][i + 1];
        else t3[i] = (L.n1 + 1) + (L.n2 + 1) + xl[2][i + 1];
    }
    const int use = 7 & ~(drop1 | drop2) & (int)mask;   // active true-null treatments
    float S = INFINITY;
    if (TABLES) {
        if (use) {
            // sort the three codes with each treatment's bit of `use` below them
            // (2 code + bit): equal codes have equal table entries, so the order
            // between them does not matter, and each sorted position carries its
            // own bit, so no permutation is tracked
            int v0 = 2 * t3[0] + (use & 1), v1 = 2 * t3[1] + ((use >> 1) & 1), v2 = 2 * t3[2] + ((use >> 2) & 1);
            int lo = min(v0, v1);
            v1 = max(v0, v1);
            v0 = lo;
            lo = min(v1, v2);
            v2 = max(v1, v2);
            v1 = lo;
            lo = min(v0, v1);
            v1 = max(v0, v1);
            v0 = lo;
            // the tables exist only when they hold at most 2^27 floats: a 32-bit index
            const float4 q = __ldg(F4 + (xl[2][0] * L.NT + triple_index(v0 >> 1, v1 >> 1, v2 >> 1)));
            // min over the counted treatments of 1 - P_i, as 1 - max P_i: x -> 1 - x
            // rounds monotonically, so the two agree bit for bit
            float pm = -1.0f;
            if (v0 & 1) pm = fmaxf(pm, q.x);
            if (v1 & 1) pm = fmaxf(pm, q.y);
            if (v2 & 1) pm = fmaxf(pm, q.z);
            S = 1.0f - pm;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if ((use >> i) & 1) {
                const float p = final_p_direct(L, C, xl[2][0], t3[i], t3[(i + 1) % 3], t3[(i + 2) % 3]);
                S = fminf(S, 1.0f - p);
            }
        }
    }
    return S;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide: index b of the bin holding the ks-th (1-indexed) element of
// hist[0..nb), and the count of elements in bins before b.  All threads call.
__device__ void find_kth(const uint32_t* hist, int nb, int ks, int* s_scan, int* s_res, int* out_b, int* out_before)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CH = (nb + BT - 1) / BT;
    const int b0 = tid * CH, b1 = min(b0 + CH, nb);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += (int)hist[b];
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_scan[warp] = incl;
    if (tid == 0) {
        s_res[0] = -1;
        s_res[1] = 0;
    }
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_scan[w];
    incl += wpre;
    const int excl = incl - local;
    if (excl < ks && ks <= incl) {
        int cum = excl;
        for (int b = b0; b < b1; ++b) {
            const int h = (int)hist[b];
            if (cum + h >= ks) {
                s_res[0] = b;
                s_res[1] = cum;
                break;
            }
            cum += h;
        }
    }
    __syncthreads();
    *out_b = s_res[0];
    *out_before = s_res[1];
    __syncthreads();
}

template <bool TABLES, bool SELECT>
__global__ void __launch_bounds__(BT, 5) k_sim_bayes4(TileArgs T, Looks L, float drop, const uint8_t* __restrict__ cnt,
                                                      int32_t NA, int32_t k_stride, int32_t K_tiles,
                                                      const uint8_t* __restrict__ D1g, const uint8_t* __restrict__ D2,
                                                      const float4* __restrict__ F4, float lambda_up, SimOut o,
                                                      uint32_t* __restrict__ keys, int32_t* __restrict__ counter,
                                                      int32_t* __restrict__ err)
{
    __shared__ uint32_t hist[2048];
    __shared__ int s_tile, s_scan[BWARP], s_res[2];
    __shared__ int s_red[5][BWARP];
    __shared__ unsigned long long s_min;   // order key of the least lambda_i of this CTA's tiles
    if (threadIdx.x == 0) s_min = ~0ull;
    extern __shared__ __align__(16) uint8_t d1s[];   // first-analysis drop table (TABLES)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    NodeConst C;
    const uint8_t* D1 = D1g;
    if (TABLES) {
        const int m = L.n1 + 1, n1t = m * m * m * m;
        for (int b = tid; b < n1t; b += BT) d1s[b] = D1g[b];
        D1 = d1s;
    } else {
        C = node_const();
    }
    uint32_t* kbuf = keys + (int64_t)blockIdx.x * k_stride;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(counter, 1);
        if (SELECT)
            for (int b = tid; b < 2048; b += BT) hist[b] = 0u;
        __syncthreads();
        const int64_t i = s_tile;
        if (i >= T.n_tiles) break;
        const int K = T.K[i];
        bool bad = (K < 1) || (K > K_tiles);
        int v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = T.center_idx[i * 4 + a];
            bad |= (v[a] < 0) || (v[a] >= T.n_axis[a]);
        }
        const int Kc = bad ? 0 : K;
        const uint32_t mask = T.null_mask[i];
        // row index of the count table for (analysis l, arm a)
        int row[3][4];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int a = 0; a < 4; ++a) row[l][a] = l * NA + T.axis_off[a] + (bad ? 0 : v[a]);
        int r_acc = 0, xs[4] = {0, 0, 0, 0};
        // four consecutive sims per thread and step: one 32-bit load per table row
        for (int k4 = tid * 4; k4 < Kc; k4 += BT * 4) {
            uint32_t w[3][4];
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    w[l][a] = __ldg(reinterpret_cast<const uint32_t*>(cnt + (int64_t)row[l][a] * k_stride + k4));
            uint32_t kq[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float S = INFINITY;
                if (k4 + j < Kc) {
                    int xl[3][4];
#pragma unroll
                    for (int l = 0; l < 3; ++l)
#pragma unroll
                        for (int a = 0; a < 4; ++a) xl[l][a] = (w[l][a] >> (8 * j)) & 0xFF;
                    S = design_stat<TABLES>(L, D1, D2, F4, C, drop, xl, mask);
                    const int rej = (S < lambda_up) ? 1 : 0;
                    r_acc += rej;
#pragma unroll
                    for (int a = 0; a < 4; ++a) xs[a] += rej * xl[2][a];   // integer multiply-add
                    if (SELECT) atomicAdd(&hist[__float_as_uint(S) >> 21], 1u);
                }
                kq[j] = __float_as_uint(S);
            }
            if (SELECT) *reinterpret_cast<uint4*>(kbuf + k4) = make_uint4(kq[0], kq[1], kq[2], kq[3]);
        }
        r_acc = warp_sum_i(r_acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) xs[a] = warp_sum_i(xs[a]);
        if (lane == 0) {
            s_red[0][warp] = r_acc;
            for (int a = 0; a < 4; ++a) s_red[1 + a][warp] = xs[a];
        }
        __syncthreads();
        double lam_i = -INFINITY;
        if (SELECT) {
            const int ks = bad ? 0 : o.ksel[i];
            if (ks >= 1) {
                // three-digit radix select (11, 11, 10 bits) over the tile's keys
                int b1, before1, b2, before2, b3, before3;
                find_kth(hist, 2048, ks, s_scan, s_res, &b1, &before1);
                for (int b = tid; b < 2048; b += BT) hist[b] = 0u;
                __syncthreads();
                for (int k = tid; k < Kc; k += BT) {
                    const uint32_t key = kbuf[k];
                    if ((int)(key >> 21) == b1) atomicAdd(&hist[(key >> 10) & 0x7FF], 1u);
                }
                __syncthreads();
                find_kth(hist, 2048, ks - before1, s_scan, s_res, &b2, &before2);
                for (int b = tid; b < 1024; b += BT) hist[b] = 0u;
                __syncthreads();
                const uint32_t pre = ((uint32_t)b1 << 11) | (uint32_t)b2;
                for (int k = tid; k < Kc; k += BT) {
                    const uint32_t key = kbuf[k];
                    if ((key >> 10) == pre) atomicAdd(&hist[key & 0x3FF], 1u);
                }
                __syncthreads();
                find_kth(hist, 1024, ks - before1 - before2, s_scan, s_res, &b3, &before3);
                lam_i = (double)__uint_as_float((pre << 10) | (uint32_t)b3);
            }
        }
        if (tid == 0) {
            if (bad) atomicOr(err, CSE_ERR_BAD_K);
            int64_t Rt = 0, X[4] = {0, 0, 0, 0};
            for (int w2 = 0; w2 < BWARP; ++w2) {
                Rt += s_red[0][w2];
                for (int a = 0; a < 4; ++a) X[a] += s_red[1 + a][w2];
            }
            if (o.R) o.R[i] = Rt;
            for (int a = 0; a < 4; ++a) {
                if (o.Xrej) o.Xrej[i * 4 + a] = X[a];
                if (o.score) {
                    const double sg = bad ? NAN : o.sig[T.axis_off[a] + v[a]];
                    o.score[i * 4 + a] = (double)X[a] - (double)L.n3 * sg * (double)Rt;
                }
            }
            if (SELECT && o.lam_tile) o.lam_tile[i] = lam_i;
            if (SELECT) s_min = min(s_min, order_key(lam_i));
        }
        __syncthreads();
    }
    queue_reset_min(counter, o.min_key, s_min, SELECT ? o.min_out : nullptr);
}

template <bool TABLES>
__global__ void k_emit_bayes4(TileArgs T, Looks L, float drop, const uint8_t* __restrict__ cnt, int32_t NA,
                              int32_t k_stride, int32_t K_tiles, const uint8_t* __restrict__ D1,
                              const uint8_t* __restrict__ D2, const float4* __restrict__ F4,
                              const int64_t* __restrict__ off, float* __restrict__ S_out, int32_t* __restrict__ err)
{
    const NodeConst C = node_const();
    for (int64_t i = blockIdx.x; i < T.n_tiles; i += gridDim.x) {
        const int K = T.K[i];
        bool bad = (K < 1) || (K > K_tiles);
        int v[4];
        for (int a = 0; a < 4; ++a) {
            v[a] = T.center_idx[i * 4 + a];
            bad |= (v[a] < 0) || (v[a] >= T.n_axis[a]);
        }
        if (bad) {
            if (threadIdx.x == 0) atomicOr(err, CSE_ERR_BAD_K);
            continue;
        }
        const uint32_t mask = T.null_mask[i];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int xl[3][4];
            for (int l = 0; l < 3; ++l)
                for (int a = 0; a < 4; ++a)
                    xl[l][a] = cnt[((int64_t)l * NA + T.axis_off[a] + v[a]) * k_stride + k];
            S_out[off[i] + k] = design_stat<TABLES>(L, D1, D2, F4, C, drop, xl, mask);
        }
    }
}

Looks make_looks(const DesignArgs& D)
{
    Looks L;
    L.n1 = D.look_n[0];
    L.n2 = D.look_n[1];
    L.n3 = D.look_n[2];
    L.S2 = (L.n1 + 1) + (L.n2 + 1);
    L.S3 = L.S2 + (L.n3 + 1);
    L.NP = L.S3 * (L.S3 + 1) / 2;
    L.NT = L.S3 * (L.S3 + 1) * (L.S3 + 2) / 6;
    return L;
}

template <bool TABLES, bool SEL>
int launch_b4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
              const SimOut& o, cudaStream_t s)
{
    auto kern = k_sim_bayes4<TABLES, SEL>;
    const Looks L = make_looks(c->D);
    const size_t smem = TABLES ? ((size_t)(L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1) + 15) / 16 * 16 : 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (SEL) {
        const size_t need = (size_t)grid * (size_t)k_stride * sizeof(uint32_t);
        if (need > c->keys_cap) {
            cudaFree(c->keys);
            c->keys = nullptr;
            c->keys_cap = 0;
            if (cudaMalloc(&c->keys, need) != cudaSuccess) {
                cudaGetLastError();
                return CSE_OOM;
            }
            c->keys_cap = need;
        }
    }
    if (SEL && o.min_out) c->min_folded = true;
    cse_prof_begin(c, KID_SIM_BAYES4, s);
    kern<<<(unsigned)grid, BT, smem, s>>>(T, L, (float)c->D.drop, c->cnt, NA, k_stride, K_tiles, c->bt_d1, c->bt_d2,
                                          c->bt_f4, lambda_float_up(lambda), o, c->keys, c->counter, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

}  // namespace

int cse_bayes4_setup(cse_ctx* c, cudaStream_t s)
{
    const Looks L = make_looks(c->D);
    const int64_t n1 = (int64_t)(L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1);
    const int64_t n2 = (int64_t)(L.n2 + 1) * L.S2 * L.S2 * L.S2;
    const int64_t n3 = (int64_t)(L.n3 + 1) * L.NT;   // float4 entries
    c->bt_tables = (n1 + n2 + 4 * n3) <= CSE_BAYES_TABLE_MAX;
    if (!c->bt_tables) return CSE_OK;   // direct evaluation per simulation
    if (cudaMalloc(&c->bt_d1, (size_t)n1) != cudaSuccess || cudaMalloc(&c->bt_d2, (size_t)n2) != cudaSuccess ||
        cudaMalloc(&c->bt_f4, (size_t)n3 * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return CSE_OOM;
    }
    const float drop = (float)c->D.drop;
    cse_prof_begin(c, KID_BAYES_TABLE, s);
    k_table_d1<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(c->bt_d1, L, drop);
    k_table_d2<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(c->bt_d2, L, drop);
    k_table_f4<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(c->bt_f4, L);
    cse_prof_end(c, s);
    c->launches += 3;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_emit_bayes4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                           const int64_t* off, float* S_out, cudaStream_t s)
{
    const int64_t grid = T.n_tiles < 4096 ? T.n_tiles : 4096;
    const Looks L = make_looks(c->D);
    if (c->bt_tables && !c->bt_direct)
        k_emit_bayes4<true><<<(unsigned)grid, 256, 0, s>>>(T, L, (float)c->D.drop, c->cnt, NA, k_stride, K_tiles,
                                                           c->bt_d1, c->bt_d2, c->bt_f4, off, S_out, c->err);
    else
        k_emit_bayes4<false><<<(unsigned)grid, 256, 0, s>>>(T, L, (float)c->D.drop, c->cnt, NA, k_stride, K_tiles,
                                                            c->bt_d1, c->bt_d2, c->bt_f4, off, S_out, c->err);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_sim_bayes4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          double lambda, const SimOut& o, cudaStream_t s)
{
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    if (c->bt_tables && !c->bt_direct) {
        return sel ? launch_b4<true, true>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                   : launch_b4<true, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
    return sel ? launch_b4<false, true>(c, T, NA, k_stride, K_tiles, lambda, o, s)
               : launch_b4<false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
}

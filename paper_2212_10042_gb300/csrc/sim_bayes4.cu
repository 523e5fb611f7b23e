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

#include <type_traits>

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

// Drop bits at the second analysis of the three treatments with codes t[0..2]
// (control: c successes of n2).  The posterior is evaluated with the treatments
// in ascending code order and the bits mapped back, so the result depends on the
// codes only as a multiset, permuted with them: treatments with equal codes hold
// equal data, and the FP32 evaluation gives them equal probabilities in either
// order.  Both the tables and the direct mode use this function.
__device__ __forceinline__ int d2_bits(const Looks& L, const NodeConst& C, float drop, int c, const int t[3])
{
    int v[3] = {4 * t[0], 4 * t[1] + 1, 4 * t[2] + 2};   // code, then treatment
    int lo = min(v[0], v[1]);
    v[1] = max(v[0], v[1]);
    v[0] = lo;
    lo = min(v[1], v[2]);
    v[2] = max(v[1], v[2]);
    v[1] = lo;
    lo = min(v[0], v[1]);
    v[1] = max(v[0], v[1]);
    v[0] = lo;
    int x[4], n[4];
    x[0] = c;
    n[0] = L.n2;
    for (int k = 0; k < 3; ++k) {
        const int code = v[k] >> 2;
        if (code <= L.n1) {
            x[k + 1] = code;
            n[k + 1] = L.n1;
        } else {
            x[k + 1] = code - (L.n1 + 1);
            n[k + 1] = L.n2;
        }
    }
    float P[3];
    posterior4_f32(x, n, C, P);
    int bits = 0;
    for (int k = 0; k < 3; ++k)
        if (P[k] < drop) bits |= 1 << (v[k] & 3);
    return bits;
}

__global__ void k_table_d2(uint8_t* __restrict__ D2, Looks L, float drop)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int S2 = L.S2;
    if (s >= (L.n2 + 1) * S2 * S2 * S2) return;
    const NodeConst C = node_const();
    const int c = s / (S2 * S2 * S2);
    const int t[3] = {(s / (S2 * S2)) % S2, (s / S2) % S2, s % S2};
    D2[s] = (uint8_t)d2_bits(L, C, drop, c, t);
}

// (a, b, z) with a <= b <= z and z (z + 1) (z + 2) / 6 + b (b + 1) / 2 + a = r.
__device__ __forceinline__ void decode_triple(int r, int* a, int* b, int* z)
{
    int zz = (int)cbrtf(6.0f * (float)r);   // largest z with z (z + 1) (z + 2) / 6 <= r
    while (zz > 0 && zz * (zz + 1) * (zz + 2) / 6 > r) --zz;
    while ((zz + 1) * (zz + 2) * (zz + 3) / 6 <= r) ++zz;
    const int r2 = r - zz * (zz + 1) * (zz + 2) / 6;
    int bb = (int)floorf((sqrtf(8.0f * r2 + 1.0f) - 1.0f) * 0.5f);   // largest b with b (b + 1) / 2 <= r2
    while (bb > 0 && bb * (bb + 1) / 2 > r2) --bb;
    while ((bb + 1) * (bb + 2) / 2 <= r2) ++bb;
    *a = r2 - bb * (bb + 1) / 2;
    *b = bb;
    *z = zz;
}

// The second-analysis drop bits over sorted code triples only, three bits an
// entry, ten entries a 32-bit word: entry e = c * NT2 + tri(a, b, z) (a <= b <= z
// < S2, NT2 = S2 (S2 + 1) (S2 + 2) / 6) sits in word e / 10 at bit 3 (e % 10)
// and holds D2[c][a][b][z], whose bit k belongs to the treatment at sorted
// position k.  By the symmetry of d2_bits this is all of D2.
__global__ void k_table_d2s(uint32_t* __restrict__ D2s, const uint8_t* __restrict__ D2, Looks L, int32_t nt2)
{
    const int64_t word = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(L.n2 + 1) * nt2;
    if (10 * word >= tot) return;
    const int S2 = L.S2;
    uint32_t out = 0u;
    for (int h = 0; h < 10; ++h) {
        const int64_t e = 10 * word + h;
        if (e >= tot) break;
        const int c = (int)(e / nt2);
        int a, b, z;
        decode_triple((int)(e % nt2), &a, &b, &z);
        out |= (uint32_t)(D2[((c * S2 + a) * S2 + b) * S2 + z] & 7) << (3 * h);
    }
    D2s[word] = out;
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
    int a, b, z;
    decode_triple((int)(s % L.NT), &a, &b, &z);
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
        bits = d2_bits(L, C, drop, xl[1][0], t2);
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

// The tabulated statistic with one trial's counts packed one arm per byte,
// Pl = [x_l0, x_l1, x_l2, x_l3] for look l (valid while every final-look code
// fits seven bits: S3 <= 128).  The same table reads as design_stat<true>, with
// the index and code arithmetic done on whole words:
// - the first-look index ((x0 m + x1) m + x2) m + x3 as (x0 m + x1) m^2 +
//   (x2 m + x3), m = n1 + 1, by two dot products of the packed bytes with packed
//   radix weights (dp4a);
// - the second-look drop bits from a table over sorted code triples held in
//   shared memory (the per-trial global gather of the full table was a fifth of
//   the kernel's time), three bits an entry, and the first-look bits four bits an
//   entry: the less shared memory the two CTAs of an SM take, the more is left
//   to L1 for the final-table gathers;
// - the codes of the next look chosen per treatment by one byte permutation:
//   byte i + 1 comes from the previous codes if treatment i was dropped, else
//   from this look's counts plus the code offset (n1 + 1, then S2).  The
//   permutation's selector is 0x7654 with bit 2 of nibble i + 1 cleared for each
//   dropped treatment: the three drop bits spread to bits 6, 10, 14 by one
//   multiply (d * 0x1240) and mask (0x4440).
struct PackedConst {
    uint32_t w1hi, w1lo, m1sq;   // first-look index weights: [m, 1, 0, 0], [0, 0, m, 1], m^2
    uint32_t off1, off2;         // code offsets on bytes 1..3: n1 + 1, S2
    int32_t nt2;                 // sorted code triples of the second analysis
};

__device__ __forceinline__ float design_stat_packed(const Looks& L, const PackedConst& Q, const uint8_t* D1,
                                                    const uint32_t* D2s, const float4* __restrict__ F4, const int* tri,
                                                    const uint32_t* perm, uint32_t P0, uint32_t P1, uint32_t P2,
                                                    uint32_t mask)
{
    // Branch-free: a trial with every treatment dropped (or none counted) runs
    // the whole sequence, every index staying within its table for any counts,
    // and gets +inf at the end; the trials of a step then form one straight
    // block that the compiler interleaves (measured: 26.8 -> 25.6 ms on the
    // refined-platten sample, with the step's bounds checks only in the tail)
    const uint32_t i1 = __dp4a(P0, Q.w1hi, 0u) * Q.m1sq + __dp4a(P0, Q.w1lo, 0u);
    const uint32_t drop1 = ((uint32_t)D1[i1 >> 1] >> ((i1 & 1u) << 2)) & 7u;   // two entries a byte
    // [x_10, codes of the three treatments at the second analysis]
    const uint32_t T2 = __byte_perm(P0, P1 + Q.off1, ((drop1 * 0x1240u) & 0x4440u) ^ 0x7654u);
    // second analysis: the codes sorted with the treatment index below them
    // (4 code + i), the sorted-triple table (k_table_d2s) in shared memory, and
    // the bits of the sorted positions mapped back to the treatments by perm
    const uint32_t V2 = ((T2 << 2) & 0xFCFCFC00u) | 0x02010000u;
    int u0 = (int)((V2 >> 8) & 0xFFu), u1 = (int)((V2 >> 16) & 0xFFu), u2 = (int)(V2 >> 24);
    int lo2 = min(u0, u1);
    u1 = max(u0, u1);
    u0 = lo2;
    lo2 = min(u1, u2);
    u2 = max(u1, u2);
    u1 = lo2;
    lo2 = min(u0, u1);
    u1 = max(u0, u1);
    u0 = lo2;
    const int e2 = (int)(T2 & 0xFFu) * Q.nt2 + tri[768 + u2] + tri[512 + u1] + (u0 >> 2);
    const uint32_t w2 = __umulhi((uint32_t)e2, 0xCCCCCCCDu) >> 3;   // e2 / 10 (exact below 2^32)
    const uint32_t nib = (D2s[w2] >> (3u * ((uint32_t)e2 - 10u * w2))) & 7u;
    const uint32_t dd = drop1 | ((perm[((u0 & 3) << 2) | (u1 & 3)] >> (3u * nib)) & 7u);
    // [x_20, codes at the final analysis]
    const uint32_t T3 = __byte_perm(T2, P2 + Q.off2, ((dd * 0x1240u) & 0x4440u) ^ 0x7654u);
    const uint32_t use = 7u & ~dd & mask;   // active true-null treatments
    // bytes 1..3: 2 code + the treatment's bit of `use`, sorted as in design_stat
    const uint32_t V = ((T3 << 1) & 0xFEFEFE00u) | ((use * 0x408100u) & 0x01010100u);
    int v0 = (int)((V >> 8) & 0xFFu), v1 = (int)((V >> 16) & 0xFFu), v2 = (int)(V >> 24);
    int lo = min(v0, v1);
    v1 = max(v0, v1);
    v0 = lo;
    lo = min(v1, v2);
    v2 = max(v1, v2);
    v1 = lo;
    lo = min(v0, v1);
    v1 = max(v0, v1);
    v0 = lo;
    // tri[v] = b (b + 1) / 2 and tri[256 + v] = c (c + 1) (c + 2) / 6 for b, c = v >> 1
    const float4 q = __ldg(F4 + ((int)(T3 & 0xFFu) * L.NT + tri[256 + v2] + tri[v1] + (v0 >> 1)));
    float pm = -1.0f;
    if (v0 & 1) pm = fmaxf(pm, q.x);
    if (v1 & 1) pm = fmaxf(pm, q.y);
    if (v2 & 1) pm = fmaxf(pm, q.z);
    return use == 0u ? INFINITY : 1.0f - pm;
}

// A streaming load of the count table that does not allocate in L1 (each count
// byte is read once per tile): L1 then keeps more final-table lines (refined
// sample 25.45 -> 25.25 ms).
__device__ __forceinline__ uint2 ld_stream2(const uint8_t* p)
{
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// Byte transpose of four words: out[j] byte a = in[a] byte j.
__device__ __forceinline__ void transpose4(const uint32_t in[4], uint32_t out[4])
{
    const uint32_t t0 = __byte_perm(in[0], in[1], 0x5140u), t1 = __byte_perm(in[2], in[3], 0x5140u);
    const uint32_t t2 = __byte_perm(in[0], in[1], 0x7362u), t3 = __byte_perm(in[2], in[3], 0x7362u);
    out[0] = __byte_perm(t0, t1, 0x5410u);
    out[1] = __byte_perm(t0, t1, 0x7632u);
    out[2] = __byte_perm(t2, t3, 0x5410u);
    out[3] = __byte_perm(t2, t3, 0x7632u);
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide: index b of the bin holding the ks-th (1-indexed) element of
// hist[0..nb), and the count of elements in bins before b.  All threads call.
template <int NTH>
__device__ void find_kth(const uint32_t* hist, int nb, int ks, int* s_scan, int* s_res, int* out_b, int* out_before)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CH = (nb + NTH - 1) / NTH;
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

// PACKED (with TABLES): the per-trial statistic by design_stat_packed, with
// 512 threads and 2 CTAs per SM (the second-look table takes 61 KB of shared
// memory per CTA; 64 registers a thread); otherwise 256 threads and 5 CTAs.
template <bool PACKED>
constexpr int b4_threads()
{
    return PACKED ? 512 : BT;
}

// Shared memory of the packed form: tri[v] = c (c + 1) / 2 and tri[256 + v] =
// c (c + 1) (c + 2) / 6 for c = v >> 1 (final-look codes with their use bit),
// tri[512 + u], tri[768 + u] the same for c = u >> 2 (second-look codes with the
// treatment index); perm[(t0 << 2) | t1] maps the drop bits of the sorted
// positions to the treatments (t0, t1, 3 - t0 - t1) at those positions: bits B
// go to (perm >> 3 B) & 7.
__device__ __forceinline__ void packed_tables(int tid, int nth, int* tri, uint32_t* perm)
{
    for (int v = tid; v < 256; v += nth) {
        const int b = v >> 1, c = v >> 2;
        tri[v] = b * (b + 1) / 2;
        tri[256 + v] = b * (b + 1) * (b + 2) / 6;
        tri[512 + v] = c * (c + 1) / 2;
        tri[768 + v] = c * (c + 1) * (c + 2) / 6;
    }
    if (tid < 16) {
        const int t0 = tid >> 2, t1 = tid & 3, t2 = 3 - t0 - t1;
        uint32_t m = 0u;
        if (t0 < 3 && t1 < 3 && t0 != t1 && t2 >= 0 && t2 < 3 && t2 != t0 && t2 != t1)
            for (uint32_t B = 0; B < 8; ++B)
                m |= ((((B & 1u) << t0) | (((B >> 1) & 1u) << t1) | (((B >> 2) & 1u) << t2))) << (3u * B);
        perm[tid] = m;
    }
}

template <bool TABLES, bool SELECT, bool PACKED>
__global__ void __launch_bounds__(b4_threads<PACKED>(), PACKED ? 2 : 5)
    k_sim_bayes4(TileArgs T, Looks L, float drop, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride,
                 int32_t K_tiles, const uint8_t* __restrict__ D1g, const uint8_t* __restrict__ D2,
                 const float4* __restrict__ F4, float lambda_up, SimOut o, uint32_t* __restrict__ keys,
                 int32_t* __restrict__ counter, int32_t* __restrict__ err, const PackedConst Q,
                 const uint32_t* __restrict__ D2sg, int32_t d1_bytes, int32_t d2s_bytes)
{
    static_assert(TABLES || !PACKED, "the packed form reads the tables");
    constexpr int NTH = b4_threads<PACKED>();
    constexpr int NW = NTH / 32;
    __shared__ uint32_t hist[2048];
    __shared__ int s_tri[PACKED ? 1024 : 1];
    __shared__ uint32_t s_perm[PACKED ? 16 : 1];
    __shared__ int s_tile, s_scan[NW], s_res[2];
    __shared__ int s_red[5][NW];
    __shared__ unsigned long long s_min;   // order key of the least lambda_i of this CTA's tiles
    if (threadIdx.x == 0) s_min = ~0ull;
    // first-analysis drop table (TABLES), then the packed form's second-analysis
    // table at d1_bytes (a multiple of 16)
    extern __shared__ __align__(16) uint8_t d1s[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    NodeConst C;
    const uint8_t* D1 = D1g;
    if (TABLES) {
        const int m = L.n1 + 1, n1t = m * m * m * m;
        if (PACKED) {   // two entries a byte
            for (int b = tid; 2 * b < n1t; b += NTH)
                d1s[b] = (uint8_t)((D1g[2 * b] & 7) | ((2 * b + 1 < n1t ? D1g[2 * b + 1] & 7 : 0) << 4));
        } else {
            for (int b = tid; b < n1t; b += NTH) d1s[b] = D1g[b];
        }
        D1 = d1s;
    } else {
        C = node_const();
    }
    const uint32_t* D2s = reinterpret_cast<const uint32_t*>(d1s + d1_bytes);
    if (PACKED) {
        packed_tables(tid, NTH, s_tri, s_perm);
        // d2s_bytes: a multiple of 16, within the global table's allocation
        for (int b = tid; b < d2s_bytes / 16; b += NTH)
            reinterpret_cast<uint4*>(d1s + d1_bytes)[b] = __ldg(reinterpret_cast<const uint4*>(D2sg) + b);
    }
    uint32_t* kbuf = keys + (int64_t)blockIdx.x * k_stride;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(counter, 1);
        if (SELECT)
            for (int b = tid; b < 2048; b += NTH) hist[b] = 0u;
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
        auto load_rows = [&](int k4, uint32_t w[3][4]) {
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    w[l][a] = __ldg(reinterpret_cast<const uint32_t*>(cnt + (int64_t)row[l][a] * k_stride + k4));
        };
        if constexpr (PACKED) {
            // eight consecutive trials per thread and step (one 8-byte load per
            // table row); the rejecting trials' final counts summed in 16-bit
            // halves (arms 0 and 2, arms 1 and 3): at most 32 steps x 8 trials x
            // 255 < 2^16 between flushes
            for (int k8 = tid * 8; k8 < Kc;) {
                uint32_t a02 = 0u, a13 = 0u;
                for (int step = 0; step < 32 && k8 < Kc; ++step, k8 += NTH * 8) {
                    uint32_t P[3][8], kq[8];
                    {
                        uint32_t wl[3][4], wh[3][4];
#pragma unroll
                        for (int l = 0; l < 3; ++l)
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                const uint2 v2 =
                                    ld_stream2(cnt + (int64_t)row[l][a] * k_stride + k8);
                                wl[l][a] = v2.x;
                                wh[l][a] = v2.y;
                            }
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            transpose4(wl[l], P[l]);
                            transpose4(wh[l], P[l] + 4);
                        }
                    }
                    auto sim8 = [&](auto full) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float S = INFINITY;
                            if (decltype(full)::value || k8 + j < Kc) {
                                S = design_stat_packed(L, Q, D1, D2s, F4, s_tri, s_perm, P[0][j], P[1][j], P[2][j],
                                                       mask);
                                const uint32_t rej = (S < lambda_up) ? 1u : 0u;
                                r_acc += (int)rej;
                                a02 += (P[2][j] & 0x00FF00FFu) * rej;
                                a13 += __byte_perm(P[2][j], 0u, 0x4341u) * rej;
                                if (SELECT) atomicAdd(&hist[__float_as_uint(S) >> 21], 1u);
                            }
                            kq[j] = __float_as_uint(S);
                        }
                    };
                    if (k8 + 8 <= Kc) sim8(std::true_type{});
                    else sim8(std::false_type{});
                    if (SELECT) {
                        *reinterpret_cast<uint4*>(kbuf + k8) = make_uint4(kq[0], kq[1], kq[2], kq[3]);
                        *reinterpret_cast<uint4*>(kbuf + k8 + 4) = make_uint4(kq[4], kq[5], kq[6], kq[7]);
                    }
                }
                xs[0] += (int)(a02 & 0xFFFFu);
                xs[2] += (int)(a02 >> 16);
                xs[1] += (int)(a13 & 0xFFFFu);
                xs[3] += (int)(a13 >> 16);
            }
        } else {
            for (int k4 = tid * 4; k4 < Kc; k4 += NTH * 4) {
                uint32_t w[3][4], kq[4];
                load_rows(k4, w);
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
                find_kth<NTH>(hist, 2048, ks, s_scan, s_res, &b1, &before1);
                for (int b = tid; b < 2048; b += NTH) hist[b] = 0u;
                __syncthreads();
                for (int k = tid; k < Kc; k += NTH) {
                    const uint32_t key = kbuf[k];
                    if ((int)(key >> 21) == b1) atomicAdd(&hist[(key >> 10) & 0x7FF], 1u);
                }
                __syncthreads();
                find_kth<NTH>(hist, 2048, ks - before1, s_scan, s_res, &b2, &before2);
                for (int b = tid; b < 1024; b += NTH) hist[b] = 0u;
                __syncthreads();
                const uint32_t pre = ((uint32_t)b1 << 11) | (uint32_t)b2;
                for (int k = tid; k < Kc; k += NTH) {
                    const uint32_t key = kbuf[k];
                    if ((key >> 10) == pre) atomicAdd(&hist[key & 0x3FF], 1u);
                }
                __syncthreads();
                find_kth<NTH>(hist, 1024, ks - before1 - before2, s_scan, s_res, &b3, &before3);
                lam_i = (double)__uint_as_float((pre << 10) | (uint32_t)b3);
            }
        }
        if (tid == 0) {
            if (bad) atomicOr(err, CSE_ERR_BAD_K);
            int64_t Rt = 0, X[4] = {0, 0, 0, 0};
            for (int w2 = 0; w2 < NW; ++w2) {
                Rt += s_red[0][w2];
                for (int a = 0; a < 4; ++a) X[a] += s_red[1 + a][w2];
            }
            if (o.R) o.R[i] = Rt;
            if (o.cp_key)   // the tile's (K, R) in the Clopper-Pearson memo, as k_cp_mark would
                o.cp_slot[i] = cp_memo_insert(((unsigned long long)(uint32_t)K << 32) | (uint32_t)Rt, o.cp_key,
                                              o.cp_cap, o.cp_list, o.cp_nkeys);
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

int64_t b4_round16(int64_t n)
{
    return (n + 15) / 16 * 16;
}

int32_t b4_nt2(const Looks& L)
{
    return L.S2 * (L.S2 + 1) * (L.S2 + 2) / 6;
}

// bytes of the sorted second-analysis table (ten entries a word), padded to 16
int64_t b4_d2s_bytes(const Looks& L)
{
    return b4_round16(4 * (((int64_t)(L.n2 + 1) * b4_nt2(L) + 9) / 10));
}

// bytes of the first-analysis table in the kernel's shared memory: a byte an
// entry, or two entries a byte in the packed form; padded to 16
int64_t b4_d1_bytes(const Looks& L, bool packed)
{
    const int64_t n = (int64_t)(L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1) * (L.n1 + 1);
    return b4_round16(packed ? (n + 1) / 2 : n);
}

template <bool TABLES, bool SEL, bool PACKED>
int launch_b4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
              const SimOut& o, cudaStream_t s)
{
    auto kern = k_sim_bayes4<TABLES, SEL, PACKED>;
    constexpr int NTH = b4_threads<PACKED>();
    const Looks L = make_looks(c->D);
    PackedConst Q{};
    if (PACKED) {
        const uint32_t m = (uint32_t)(L.n1 + 1), s2 = (uint32_t)L.S2;
        Q.w1hi = m | (1u << 8);
        Q.w1lo = (m << 16) | (1u << 24);
        Q.m1sq = m * m;
        Q.off1 = m * 0x01010100u;
        Q.off2 = s2 * 0x01010100u;
        Q.nt2 = b4_nt2(L);
    }
    const int32_t d1_bytes = TABLES ? (int32_t)b4_d1_bytes(L, PACKED) : 0;
    const int32_t d2s_bytes = PACKED ? (int32_t)b4_d2s_bytes(L) : 0;
    const size_t smem = (size_t)d1_bytes + (size_t)d2s_bytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTH, smem) != cudaSuccess || per_sm < 1) {
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
    if (o.cp_key) c->cp_marked = true;
    cse_prof_begin(c, KID_SIM_BAYES4, s);
    kern<<<(unsigned)grid, NTH, smem, s>>>(T, L, (float)c->D.drop, c->cnt, NA, k_stride, K_tiles, c->bt_d1, c->bt_d2,
                                           c->bt_f4, lambda_float_up(lambda), o, c->keys, c->counter, c->err, Q,
                                           c->bt_d2s, d1_bytes, d2s_bytes);
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
    // the packed per-trial form: every final-look code in seven bits, second-look
    // codes in six, and both shared-memory tables within 96 KB (2 CTAs per SM)
    const int64_t d2s = b4_d2s_bytes(L);
    c->bt_packed = L.S3 <= 128 && L.S2 <= 64 && b4_d1_bytes(L, true) + d2s <= 96 * 1024;
    if (c->bt_packed) {
        if (cudaMalloc(&c->bt_d2s, (size_t)d2s) != cudaSuccess) {
            cudaGetLastError();
            return CSE_OOM;
        }
        const int64_t nw = ((int64_t)(L.n2 + 1) * b4_nt2(L) + 9) / 10;
        if (cudaMemsetAsync(c->bt_d2s, 0, (size_t)d2s, s) != cudaSuccess) {
            cudaGetLastError();
            return CSE_CUDA_ERROR;
        }
        k_table_d2s<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(c->bt_d2s, c->bt_d2, L, b4_nt2(L));
        c->launches += 1;
    }
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
        if (c->bt_packed)
            return sel ? launch_b4<true, true, true>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                       : launch_b4<true, false, true>(c, T, NA, k_stride, K_tiles, lambda, o, s);
        return sel ? launch_b4<true, true, false>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                   : launch_b4<true, false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
    return sel ? launch_b4<false, true, false>(c, T, NA, k_stride, K_tiles, lambda, o, s)
               : launch_b4<false, false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
}

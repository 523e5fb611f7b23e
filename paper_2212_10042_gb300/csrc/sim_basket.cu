// sim_basket.cu -- the Bayesian basket trial of Sec. 10.1: four arms of n patients
// (n = 35 in the paper), one analysis, and the hierarchical model
//   theta_i ~ N(mu, s2), mu ~ N(-1.34, 100), s2 ~ InvGamma(0.0005, 0.000005)
// on the offset log-odds theta_i = logit(p_i) - t_i, where t_i is the logit of
// arm i's null response rate.  Each arm's likelihood is replaced by the normal
// approximation of its empirical logit (x + 1/2 successes, n - x + 1/2
// failures), s2 is integrated on the 16 log-spaced nodes shared with the
// four-arm selection design, mu and the thetas exactly.  Arm i is rejected when
// P(theta_i > 0 | x) > 1 - lambda (lambda = 0.15: the 85% rule); the FWER
// statistic of a tile is S = min over the tile's null arms of 1 - P_i.
//
// The posterior depends on a trial only through its four success counts, so the
// context tabulates Q_i = 1 - P_i in FP32 over all (n + 1)^4 count states once
// (a float4 per state, 27 MB for n = 35, L2-resident).  A simulated trial then
// costs four count-byte reads (coalesced) and one 16-byte gather.  The direct
// mode (plain path) evaluates the same FP32 function per trial instead.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "cse_internal.cuh"

namespace {

constexpr int BT = 256;          // threads of the simulation kernel
constexpr int BWARP = BT / 32;
constexpr int SPT = 8;           // consecutive sims per thread and step (one 8-byte count load per arm)

struct Basket {
    int n;        // patients per arm
    int m;        // n + 1: count states per arm
    float t[4];   // null logits t_i
};

// Q_i = 1 - P(theta_i > 0 | x) for the four arms, FP32.  Not inlined, so the
// table builder and the direct mode run the same instruction sequence.
__device__ __noinline__ void basket_q_f32(const int* x, const Basket& B, const NodeConst& C, float* Q)
{
    const float MU0 = -1.34f, TAU2 = 100.0f;
    float th[4], s2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float xs = (float)x[i] + 0.5f, fs = (float)(B.n - x[i]) + 0.5f;
        th[i] = logf(xs / fs) - B.t[i];
        s2[i] = 1.0f / xs + 1.0f / fs;
    }
    float lw[kBayesNodes], qj[kBayesNodes][4];
    float mx = -INFINITY;
#pragma unroll 4
    for (int j = 0; j < kBayesNodes; ++j) {
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
        // N(theta_hat; mu0 1, s2 I + diag(s_i^2) + 100 11') by the rank-one update
        const float prec = 1.0f / TAU2 + W;
        const float quad = Srr - Sr * Sr / prec;
        const float logdet = logf(prod * (1.0f + TAU2 * W));
        lw[j] = C.lprior[j] - 0.5f * logdet - 0.5f * quad;
        mx = fmaxf(mx, lw[j]);
        const float mmu = (MU0 / TAU2 + Sth) / prec;
        const float vmu = 1.0f / prec;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // theta_i | mu, s2, x ~ N((1 - c) th_i + c mu, s_i^2 s2 / (s_i^2 + s2)), c = s_i^2 / (s_i^2 + s2);
            // mu integrated over N(mmu, vmu)
            const float c = s2[i] * w[i];
            const float v = s2[i] * sg * w[i] + c * c * vmu;
            const float e = (1.0f - c) * th[i] + c * mmu;
            qj[j][i] = normcdff(-e * rsqrtf(v));   // 1 - P(theta_i > 0) without the cancellation
        }
    }
    float Z = 0.f, a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kBayesNodes; ++j) {
        const float wj = expf(lw[j] - mx);
        Z += wj;
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] += wj * qj[j][i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) Q[i] = a[i] / Z;
}

__global__ void k_table_basket(float4* __restrict__ Qt, Basket B)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = B.m;
    if (s >= m * m * m * m) return;
    const NodeConst C = node_const();
    const int x[4] = {s / (m * m * m), (s / (m * m)) % m, (s / m) % m, s % m};
    float Q[4];
    basket_q_f32(x, B, C, Q);
    Qt[s] = make_float4(Q[0], Q[1], Q[2], Q[3]);
}

// S of one trial: min over the null arms in `mask` of Q_i (+inf when none).
__device__ __forceinline__ float masked_min(const float4& q, uint32_t mask)
{
    float S = INFINITY;
    if (mask & 1u) S = fminf(S, q.x);
    if (mask & 2u) S = fminf(S, q.y);
    if (mask & 4u) S = fminf(S, q.z);
    if (mask & 8u) S = fminf(S, q.w);
    return S;
}

template <bool TABLE>
__device__ __forceinline__ float4 state_q(const float4* __restrict__ Qt, const Basket& B, const NodeConst& C,
                                          const int* x)
{
    if (TABLE) return __ldg(Qt + ((x[0] * B.m + x[1]) * B.m + x[2]) * B.m + x[3]);
    float Q[4];
    basket_q_f32(x, B, C, Q);
    return make_float4(Q[0], Q[1], Q[2], Q[3]);
}

__device__ __forceinline__ int basket_warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Persistent: each CTA takes tiles from the work queue; the tile's K sims are
// spread over the block, SPT consecutive sims per thread and step, their eight
// gathers issued before any is used.  SELECT adds the per-tile order statistic
// lambda_i = S_(ksel_i) by a three-digit radix select (11, 11, 10 bits of the
// FP32 keys, which order like the non-negative S) over the keys the CTA stored.
template <bool TABLE, bool SELECT>
__global__ void __launch_bounds__(BT, 4) k_sim_basket(TileArgs T, Basket B, const uint8_t* __restrict__ cnt,
                                                      int32_t k_stride, int32_t K_tiles,
                                                      const float4* __restrict__ Qt, float lambda_up, SimOut o,
                                                      uint32_t* __restrict__ keys, int32_t* __restrict__ counter,
                                                      int32_t* __restrict__ err)
{
    __shared__ uint32_t hist[2048];
    __shared__ int s_tile, s_scan[BWARP], s_res[2];
    __shared__ int s_red[5][BWARP];
    __shared__ unsigned long long s_min;   // order key of the least lambda_i of this CTA's tiles
    if (threadIdx.x == 0) s_min = ~0ull;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    NodeConst C;
    if (!TABLE) C = node_const();
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
        const uint8_t* rowp[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) rowp[a] = cnt + (int64_t)(T.axis_off[a] + (bad ? 0 : v[a])) * k_stride;
        int r_acc = 0, xs[4] = {0, 0, 0, 0};
        if constexpr (TABLE) {
            // full steps without per-trial bounds checks, the tail step with them:
            // straight-line work for the eight trials (16^4 grid: 4.08 -> 3.66 ms)
            auto step8 = [&](int k8, auto full) {
                // k8 + SPT <= k_stride (k_stride is a multiple of 16): the loads stay in the row
                uint2 w[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) w[a] = __ldg(reinterpret_cast<const uint2*>(rowp[a] + k8));
                float4 q[SPT];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    q[j] = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
                    if (decltype(full)::value || k8 + j < Kc) {
                        int x[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            x[a] = min((int)(((j < 4 ? w[a].x : w[a].y) >> (8 * (j & 3))) & 0xFFu), B.n);
                        q[j] = state_q<TABLE>(Qt, B, C, x);
                    }
                }
                uint32_t kq[SPT];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    float S = INFINITY;
                    if (decltype(full)::value || k8 + j < Kc) {
                        S = masked_min(q[j], mask);
                        const int rej = (S < lambda_up) ? 1 : 0;
                        r_acc += rej;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int x = min((int)(((j < 4 ? w[a].x : w[a].y) >> (8 * (j & 3))) & 0xFFu), B.n);
                            xs[a] += rej ? x : 0;
                        }
                        if (SELECT) atomicAdd(&hist[__float_as_uint(S) >> 21], 1u);
                    }
                    kq[j] = __float_as_uint(S);
                }
                if (SELECT) {
                    *reinterpret_cast<uint4*>(kbuf + k8) = make_uint4(kq[0], kq[1], kq[2], kq[3]);
                    *reinterpret_cast<uint4*>(kbuf + k8 + 4) = make_uint4(kq[4], kq[5], kq[6], kq[7]);
                }
            };
            int k8 = tid * SPT;
            for (; k8 + SPT <= Kc; k8 += BT * SPT) step8(k8, std::true_type{});
            if (k8 < Kc) step8(k8, std::false_type{});
        } else {
            for (int k8 = tid * SPT; k8 < Kc; k8 += BT * SPT) {
                // k8 + SPT <= k_stride (k_stride is a multiple of 16): the loads stay in the row
                uint2 w[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) w[a] = __ldg(reinterpret_cast<const uint2*>(rowp[a] + k8));
                float4 q[SPT];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    q[j] = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
                    if (k8 + j < Kc) {
                        int x[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            x[a] = min((int)(((j < 4 ? w[a].x : w[a].y) >> (8 * (j & 3))) & 0xFFu), B.n);
                        q[j] = state_q<TABLE>(Qt, B, C, x);
                    }
                }
                uint32_t kq[SPT];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    float S = INFINITY;
                    if (k8 + j < Kc) {
                        S = masked_min(q[j], mask);
                        const int rej = (S < lambda_up) ? 1 : 0;
                        r_acc += rej;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int x = min((int)(((j < 4 ? w[a].x : w[a].y) >> (8 * (j & 3))) & 0xFFu), B.n);
                            xs[a] += rej ? x : 0;
                        }
                        if (SELECT) atomicAdd(&hist[__float_as_uint(S) >> 21], 1u);
                    }
                    kq[j] = __float_as_uint(S);
                }
                if (SELECT) {
                    *reinterpret_cast<uint4*>(kbuf + k8) = make_uint4(kq[0], kq[1], kq[2], kq[3]);
                    *reinterpret_cast<uint4*>(kbuf + k8 + 4) = make_uint4(kq[4], kq[5], kq[6], kq[7]);
                }
            }
        }
        r_acc = basket_warp_sum(r_acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) xs[a] = basket_warp_sum(xs[a]);
        if (lane == 0) {
            s_red[0][warp] = r_acc;
            for (int a = 0; a < 4; ++a) s_red[1 + a][warp] = xs[a];
        }
        __syncthreads();
        double lam_i = -INFINITY;
        if (SELECT) {
            const int ks = bad ? 0 : o.ksel[i];
            if (ks >= 1) {
                int before1, before2, before3;
                const int b1 = block_find_kth<BT>(hist, 2048, ks, s_scan, s_res, &before1);
                for (int b = tid; b < 2048; b += BT) hist[b] = 0u;
                __syncthreads();
                for (int k = tid; k < Kc; k += BT) {
                    const uint32_t key = kbuf[k];
                    if ((int)(key >> 21) == b1) atomicAdd(&hist[(key >> 10) & 0x7FF], 1u);
                }
                const int b2 = block_find_kth<BT>(hist, 2048, ks - before1, s_scan, s_res, &before2);
                for (int b = tid; b < 1024; b += BT) hist[b] = 0u;
                __syncthreads();
                const uint32_t pre = ((uint32_t)b1 << 11) | (uint32_t)b2;
                for (int k = tid; k < Kc; k += BT) {
                    const uint32_t key = kbuf[k];
                    if ((key >> 10) == pre) atomicAdd(&hist[key & 0x3FF], 1u);
                }
                const int b3 = block_find_kth<BT>(hist, 1024, ks - before1 - before2, s_scan, s_res, &before3);
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
                    o.score[i * 4 + a] = (double)X[a] - (double)B.n * sg * (double)Rt;
                }
            }
            if (SELECT && o.lam_tile) o.lam_tile[i] = lam_i;
            if (SELECT) s_min = min(s_min, order_key(lam_i));
        }
        __syncthreads();
    }
    queue_reset_min(counter, o.min_key, s_min, SELECT ? o.min_out : nullptr);
}

template <bool TABLE>
__global__ void k_emit_basket(TileArgs T, Basket B, const uint8_t* __restrict__ cnt, int32_t k_stride,
                              int32_t K_tiles, const float4* __restrict__ Qt, const int64_t* __restrict__ off,
                              float* __restrict__ S_out, int32_t* __restrict__ err)
{
    NodeConst C;
    if (!TABLE) C = node_const();
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
            int x[4];
            for (int a = 0; a < 4; ++a)
                x[a] = min((int)cnt[(int64_t)(T.axis_off[a] + v[a]) * k_stride + k], B.n);
            S_out[off[i] + k] = masked_min(state_q<TABLE>(Qt, B, C, x), mask);
        }
    }
}

Basket make_basket(const DesignArgs& D)
{
    Basket B;
    B.n = D.look_n[0];
    B.m = B.n + 1;
    for (int a = 0; a < 4; ++a) B.t[a] = (float)D.tnull[a];
    return B;
}

template <bool TABLE, bool SEL>
int launch_basket(cse_ctx* c, const TileArgs& T, int32_t k_stride, int32_t K_tiles, double lambda, const SimOut& o,
                  cudaStream_t s)
{
    auto kern = k_sim_basket<TABLE, SEL>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, 0) != cudaSuccess || per_sm < 1) {
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
    cse_prof_begin(c, KID_SIM_BASKET, s);
    kern<<<(unsigned)grid, BT, 0, s>>>(T, make_basket(c->D), c->cnt, k_stride, K_tiles, c->bk_q,
                                      lambda_float_up(lambda), o, c->keys, c->counter, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

}  // namespace

int cse_basket_setup(cse_ctx* c, cudaStream_t s)
{
    const Basket B = make_basket(c->D);
    const int64_t states = (int64_t)B.m * B.m * B.m * B.m;
    c->bt_tables = states <= CSE_BAYES_TABLE_MAX;
    if (!c->bt_tables) return CSE_OK;   // direct evaluation per simulation
    if (cudaMalloc(&c->bk_q, (size_t)states * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return CSE_OOM;
    }
    cse_prof_begin(c, KID_BASKET_TABLE, s);
    k_table_basket<<<(unsigned)((states + 255) / 256), 256, 0, s>>>(c->bk_q, B);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_emit_basket(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                           const int64_t* off, float* S_out, cudaStream_t s)
{
    (void)NA;
    const int64_t grid = T.n_tiles < 4096 ? T.n_tiles : 4096;
    const Basket B = make_basket(c->D);
    if (c->bt_tables && !c->bt_direct)
        k_emit_basket<true><<<(unsigned)grid, 256, 0, s>>>(T, B, c->cnt, k_stride, K_tiles, c->bk_q, off, S_out,
                                                           c->err);
    else
        k_emit_basket<false><<<(unsigned)grid, 256, 0, s>>>(T, B, c->cnt, k_stride, K_tiles, c->bk_q, off, S_out,
                                                            c->err);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_sim_basket(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          double lambda, const SimOut& o, cudaStream_t s)
{
    (void)NA;
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    if (c->bt_tables && !c->bt_direct)
        return sel ? launch_basket<true, true>(c, T, k_stride, K_tiles, lambda, o, s)
                   : launch_basket<true, false>(c, T, k_stride, K_tiles, lambda, o, s);
    return sel ? launch_basket<false, true>(c, T, k_stride, K_tiles, lambda, o, s)
               : launch_basket<false, false>(c, T, k_stride, K_tiles, lambda, o, s);
}

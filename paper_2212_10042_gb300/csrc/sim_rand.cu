// sim_rand.cu -- the randomised z-tests (Sec. 7, after Thm. calibration): the
// statistic is the pair (S, w) with w the sim's independent tie-break word, the
// threshold the pair (lambda, c), compared lexicographically:
//   reject iff S < lambda, or S = lambda and w < c          (c = 0: S < lambda).
//
// k_sim_rand processes one tile per CTA iteration (persistent, atomic work
// queue).  Per sim: the final-look counts from the axis count table, the cell's
// rank from a shared copy of the rank table (rank = number of cells with a
// smaller statistic, so S < lambda iff rank < rho and S = lambda iff rank = rho
// when lambda is a table value), the sim's word when its cell ties lambda.
// With calibration on (SELECT) each sim also adds to a per-rank histogram;
// after the pass the k-th smallest pair is found in two steps: the rank r* of
// the k-th smallest statistic (block-wide prefix search of the histogram), then
// the m-th smallest word among the sims of rank r* (m = k - number of sims below
// r*), gathered into a per-CTA buffer and radix-selected (11, 11, 10 bits).
#include <cuda_runtime.h>
#include <math.h>

#include "cse_internal.cuh"

namespace {

constexpr int kRandThreads = 256;

__device__ __forceinline__ int rand_warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool TWO_ARM, bool SELECT, int NT>
__global__ void __launch_bounds__(NT) k_sim_rand(
    TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride, int32_t K_tiles,
    const uint16_t* __restrict__ rank_g, const float* __restrict__ S_g, const float* __restrict__ vor_g,
    int32_t n_cells, int32_t n1p, double lambda, uint32_t c_thr, const uint32_t* __restrict__ W, SimOut o,
    uint32_t* __restrict__ c_tile, uint32_t* __restrict__ tbuf, int32_t* __restrict__ counter,
    int32_t* __restrict__ err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int NW = NT / 32;
    // the rank histogram doubles as the radix-select digit histogram (2048 bins)
    const int hw = SELECT ? max(n_cells, 2048) : 0;
    uint32_t* hist = smem;                                                  // [hw]
    uint16_t* rt = reinterpret_cast<uint16_t*>(smem + hw);                  // [n_cells]
    __shared__ int s_tile, s_rho, s_eq, s_g;
    __shared__ int s_red[3][NW];
    __shared__ int s_scan[NW];
    __shared__ int s_res[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_rho = 0;
        s_eq = 0;
    }
    __syncthreads();
    int rho = 0, eq = 0;
    for (int c = tid; c < hw; c += NT) hist[c] = 0u;
    for (int c = tid; c < n_cells; c += NT) {
        rt[c] = rank_g[c];
        const double s = (double)S_g[c];
        rho += (s < lambda) ? 1 : 0;
        eq |= (s == lambda) ? 1 : 0;
    }
    rho = rand_warp_sum(rho);
    eq = __any_sync(0xffffffffu, eq) ? 1 : 0;
    if (lane == 0) {
        atomicAdd(&s_rho, rho);
        if (eq) atomicOr(&s_eq, 1);
    }
    __syncthreads();
    rho = s_rho;
    // rank of the cells that tie lambda (-1: lambda is not a table value)
    const int tie_rank = (s_eq && c_thr > 0u) ? rho : -1;

    const int last = D.n_looks - 1;
    const int d = T.d;
    uint32_t* buf = tbuf + (int64_t)blockIdx.x * K_tiles;
    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(counter, 1);
            s_g = 0;
        }
        __syncthreads();
        const int64_t i = s_tile;
        if (i >= T.n_tiles) break;
        const int K = T.K[i];
        const int v0 = T.center_idx[i * d + 0];
        const int v1 = TWO_ARM ? T.center_idx[i * d + 1] : 0;
        const bool badK = (K < 1) || (K > K_tiles) || v0 < 0 || v0 >= T.n_axis[0] ||
                          (TWO_ARM && (v1 < 0 || v1 >= T.n_axis[1]));
        const int Kc = badK ? 0 : K;
        const int a0 = T.axis_off[0] + (badK ? 0 : v0);
        const int a1 = TWO_ARM ? T.axis_off[1] + (badK ? 0 : v1) : 0;
        const uint8_t* c0 = cnt + ((int64_t)last * NA + a0) * k_stride;
        const uint8_t* c1 = TWO_ARM ? cnt + ((int64_t)last * NA + a1) * k_stride : c0;

        int r_acc = 0, x0_acc = 0, x1_acc = 0;
        for (int k = tid; k < Kc; k += NT) {
            const int x0 = c0[k];
            const int x1 = TWO_ARM ? (int)c1[k] : 0;
            const int cell = TWO_ARM ? x0 * n1p + x1 : x0;
            const int r = rt[cell];
            int rej = r < rho;
            if (r == tie_rank) rej = W[k] < c_thr;
            r_acc += rej;
            x0_acc += rej * x0;
            x1_acc += rej * x1;
            if (SELECT) atomicAdd(&hist[r], 1u);
        }
        r_acc = rand_warp_sum(r_acc);
        x0_acc = rand_warp_sum(x0_acc);
        if (TWO_ARM) x1_acc = rand_warp_sum(x1_acc);
        if (lane == 0) {
            s_red[0][warp] = r_acc;
            s_red[1][warp] = x0_acc;
            s_red[2][warp] = x1_acc;
        }
        __syncthreads();

        double lam_i = -INFINITY;
        uint32_t c_i = 0u;
        if (SELECT) {
            const int ks = badK ? 0 : o.ksel[i];
            int before = 0;
            const int rstar = block_find_kth<NT>(hist, n_cells, ks, s_scan, s_res, &before);
            // clear the rank histogram for the next tile (read by nobody after the search)
            for (int c = tid; c < n_cells; c += NT) hist[c] = 0u;
            if (rstar >= 0) {
                // gather the words of the sims of rank r*
                for (int k = tid; k < Kc; k += NT) {
                    const int x0 = c0[k];
                    const int cell = TWO_ARM ? x0 * n1p + (int)c1[k] : x0;
                    if (rt[cell] == rstar) buf[atomicAdd(&s_g, 1)] = W[k];
                }
                __syncthreads();
                const int g = s_g;
                int m = ks - before;   // 1 <= m <= g
                // radix select of the m-th smallest word: digits of 11, 11, 10 bits,
                // counted in the (cleared) histogram's first 2048 words
                uint32_t prefix = 0u, pmask = 0u;
                for (int pass = 0; pass < 3; ++pass) {
                    const int sh = (pass == 0) ? 21 : (pass == 1) ? 10 : 0;
                    const int nb = (pass < 2) ? 2048 : 1024;
                    for (int k = tid; k < g; k += NT) {
                        const uint32_t v = buf[k];
                        if ((v & pmask) == prefix) atomicAdd(&hist[(v >> sh) & (uint32_t)(nb - 1)], 1u);
                    }
                    __syncthreads();
                    int bef = 0;
                    const int digit = block_find_kth<NT>(hist, nb, m, s_scan, s_res, &bef);
                    for (int b = tid; b < nb; b += NT) hist[b] = 0u;
                    __syncthreads();   // cleared before the next pass counts
                    if (digit < 0) {   // cannot happen: the group holds m words
                        if (tid == 0) atomicOr(err, CSE_ERR_BAD_K);
                        break;
                    }
                    m -= bef;
                    prefix |= (uint32_t)digit << sh;
                    pmask |= (uint32_t)(nb - 1) << sh;
                }
                lam_i = (double)vor_g[rstar];
                c_i = prefix;
            }
            __syncthreads();
        }
        if (tid == 0) {
            if (badK) atomicOr(err, CSE_ERR_BAD_K);
            int64_t Rt = 0, X0 = 0, X1 = 0;
            for (int w = 0; w < NW; ++w) {
                Rt += s_red[0][w];
                X0 += s_red[1][w];
                X1 += s_red[2][w];
            }
            if (o.R) o.R[i] = Rt;
            if (o.Xrej) {
                o.Xrej[i * d + 0] = X0;
                if (TWO_ARM) o.Xrej[i * d + 1] = X1;
            }
            if (o.score) {
                const double nm = (double)D.n_max;
                const double s0 = badK ? NAN : o.sig[a0];
                o.score[i * d + 0] = (double)X0 - nm * s0 * (double)Rt;
                if (TWO_ARM) {
                    const double s1 = badK ? NAN : o.sig[a1];
                    o.score[i * d + 1] = (double)X1 - nm * s1 * (double)Rt;
                }
            }
            if (SELECT) {
                if (o.lam_tile) o.lam_tile[i] = lam_i;
                if (c_tile) c_tile[i] = c_i;
            }
        }
        __syncthreads();
    }
}

// Lexicographic minimum of (lambda_i, c_i) over tiles: the key
// (order key of float(lambda_i)) << 32 | c_i orders the pairs; lambda_i are
// FP32 table values or -inf, so the float conversion is exact.
__device__ __forceinline__ uint32_t order_key32(float x)
{
    const uint32_t b = __float_as_uint(x);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float order_unkey32(uint32_t k)
{
    return __uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void __launch_bounds__(256) k_min_pair(const double* __restrict__ lam, const uint32_t* __restrict__ c,
                                                  int64_t n, double* __restrict__ lam_out,
                                                  uint32_t* __restrict__ c_out, unsigned long long* __restrict__ key,
                                                  unsigned int* __restrict__ ticket)
{
    __shared__ unsigned long long red[8];
    __shared__ bool last;
    unsigned long long m = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = min(m, ((unsigned long long)order_key32((float)lam[i]) << 32) | c[i]);
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
        *lam_out = (k == ~0ull) ? INFINITY : (double)order_unkey32((uint32_t)(k >> 32));
        *c_out = (k == ~0ull) ? 0u : (uint32_t)k;
        *ticket = 0u;
    }
}

template <bool TWO, bool SEL>
size_t rand_smem(const cse_ctx* c)
{
    const size_t hw = SEL ? (size_t)(c->n_cells > 2048 ? c->n_cells : 2048) : 0;
    return hw * 4 + ((size_t)c->n_cells * 2 + 15) / 16 * 16;
}

template <bool TWO, bool SEL>
int launch_rand(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                uint32_t c_thr, const SimOut& o, uint32_t* c_tile, cudaStream_t s)
{
    auto kern = k_sim_rand<TWO, SEL, kRandThreads>;
    const size_t smem = rand_smem<TWO, SEL>(c);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRandThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) grid = 1;
    if (SEL) {   // per-CTA buffer of tie-group words
        const size_t need = sizeof(uint32_t) * (size_t)grid * (size_t)K_tiles;
        if (need > c->tbuf_cap) {
            cudaFree(c->tbuf);
            c->tbuf = nullptr;
            c->tbuf_cap = 0;
            if (cudaMalloc(&c->tbuf, need) != cudaSuccess) {
                cudaGetLastError();
                return CSE_OOM;
            }
            c->tbuf_cap = need;
        }
    }
    if (cudaMemsetAsync(c->counter, 0, sizeof(int32_t), s) != cudaSuccess) return CSE_CUDA_ERROR;
    cse_prof_begin(c, KID_SIM_ZTEST, s);
    kern<<<(unsigned)grid, kRandThreads, smem, s>>>(T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab,
                                                    c->val_of_rank, c->n_cells, c->n1p, lambda, c_thr, c->tb, o,
                                                    c_tile, c->tbuf, c->counter, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

}  // namespace

int cse_launch_sim_rand(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                        uint32_t c_thr, const SimOut& o, uint32_t* c_tile, cudaStream_t s)
{
    if (c->D.stat != CSE_STAT_ONE_ARM_Z && c->D.stat != CSE_STAT_TWO_ARM_POOLED_Z) return CSE_UNSUPPORTED_DESIGN;
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    if (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z)
        return sel ? launch_rand<true, true>(c, T, NA, k_stride, K_tiles, lambda, c_thr, o, c_tile, s)
                   : launch_rand<true, false>(c, T, NA, k_stride, K_tiles, lambda, c_thr, o, c_tile, s);
    return sel ? launch_rand<false, true>(c, T, NA, k_stride, K_tiles, lambda, c_thr, o, c_tile, s)
               : launch_rand<false, false>(c, T, NA, k_stride, K_tiles, lambda, c_thr, o, c_tile, s);
}

int cse_launch_min_pair(cse_ctx* c, const double* lam_tile, const uint32_t* c_tile, int64_t n, double* lam_out,
                        uint32_t* c_out, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 2 * (int64_t)c->num_sms) blocks = 2 * (int64_t)c->num_sms;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(c->min_key, 0xFF, sizeof(unsigned long long), s) != cudaSuccess) return CSE_CUDA_ERROR;
    cse_prof_begin(c, KID_MIN, s);
    k_min_pair<<<(unsigned)blocks, 256, 0, s>>>(lam_tile, c_tile, n, lam_out, c_out, c->min_key, c->min_ticket);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

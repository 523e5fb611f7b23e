// sim_ztest.cu -- persistent simulation kernel for the one- and two-arm z-tests.
//
// For every tile i and sim k < K_i (Sec. 6.1 / 7.1): success counts x_a are read
// from the axis count table (a binary search on the sorted CRN uniforms, done
// once per distinct axis value and sim), the FP32 statistic's rank is looked up
// in a shared-memory table, the design rejects iff S < lambda (rank < rank of
// lambda), and the tile accumulates
//   R = sum_k 1{rej},  Xrej_a = sum_k 1{rej} x_a            (exact integers),
//   score_a = Xrej_a - n_max sigmoid(theta_a) R              (FP64, Ex. exp-fam).
// With calibration on, every sim's rank also goes into a shared-memory
// histogram, and the k_i-th smallest statistic (Eq. calibrated-threshold) is read
// off a block-wide prefix scan of that histogram.
//
// One CTA processes one tile at a time and pulls the next tile index from a
// global counter (persistent, load-balanced over uneven K_i).
#include <cuda_runtime.h>
#include <math.h>

#include "cse_internal.cuh"

namespace {

// threads per CTA of the simulation kernel: chosen per context by the autotuner
constexpr int kThreadOptions[3] = {128, 256, 512};

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool PACKED>
__device__ __forceinline__ int bin_count(const uint32_t* hist, int b)
{
    if (PACKED) return (int)((hist[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu);
    return (int)hist[b];
}

// One tile per CTA iteration.  PACKED: the rank histogram holds two 16-bit
// counters per word (valid while K < 65536), halving its shared memory.
// DIRECT (plain comparison path): every (tile, sim, arm) count is its own binary
// search in the sorted uniforms instead of a read of the axis count table.
template <bool TWO_ARM, bool SELECT, bool PACKED, bool DIRECT, int NT>
__global__ void __launch_bounds__(NT) k_sim_ztest(
    TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride, int32_t K_tiles,
    const uint16_t* __restrict__ rank_g, const float* __restrict__ S_g, const float* __restrict__ vor_g,
    int32_t n_cells, int32_t n1p, float lambda_up, SimOut o, int32_t* __restrict__ counter,
    int32_t* __restrict__ err, const uint32_t* __restrict__ U, const uint32_t* __restrict__ thr, int32_t K_max_ctx)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int n_words = SELECT ? (PACKED ? (n_cells + 1) / 2 : n_cells) : 0;
    uint32_t* hist = smem;                                               // [n_words]
    uint16_t* rt = reinterpret_cast<uint16_t*>(smem + ((n_words + 3) & ~3));   // [n_cells]
    __shared__ int s_tile;
    __shared__ int s_rho;
    __shared__ int s_red[3][(NT / 32)];
    __shared__ int s_scan[(NT / 32)];
    __shared__ int s_pick;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_rho = 0;
    __syncthreads();
    int rho = 0;
    for (int c = tid; c < n_cells; c += NT) {
        rt[c] = rank_g[c];
        rho += (S_g[c] < lambda_up) ? 1 : 0;
    }
    rho = warp_sum(rho);
    if (lane == 0) atomicAdd(&s_rho, rho);
    __syncthreads();
    rho = s_rho;

    const int last = D.n_looks - 1;
    const int d = T.d;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(counter, 1);
        if (SELECT) {
            for (int c = tid; c < n_words; c += NT) hist[c] = 0u;
        }
        __syncthreads();
        const int64_t i = s_tile;
        if (i >= T.n_tiles) break;
        const int K = T.K[i];
        const int v0 = T.center_idx[i * d + 0];
        const int v1 = TWO_ARM ? T.center_idx[i * d + 1] : 0;
        // device-side argument checks: K_i in [1, K_max of the set], axis indices in range
        const bool badK = (K < 1) || (K > K_tiles) || v0 < 0 || v0 >= T.n_axis[0] ||
                          (TWO_ARM && (v1 < 0 || v1 >= T.n_axis[1]));
        const int Kc = badK ? 0 : K;
        const uint8_t* c0 = cnt + ((int64_t)last * NA + T.axis_off[0] + (badK ? 0 : v0)) * k_stride;
        const uint8_t* c1 = c0;
        if (TWO_ARM) c1 = cnt + ((int64_t)last * NA + T.axis_off[1] + (badK ? 0 : v1)) * k_stride;
        int r_acc = 0, x0_acc = 0, x1_acc = 0;
        if (DIRECT) {
            const int nm = D.n_max;
            const uint32_t t0 = badK ? 0u : thr[T.axis_off[0] + v0];
            const uint32_t t1 = (TWO_ARM && !badK) ? thr[T.axis_off[1] + v1] : 0u;
            for (int k = tid; k < Kc; k += NT) {
                const int x0 = count_below(U + (int64_t)k * nm, nm, t0);
                const int x1 = TWO_ARM ? count_below(U + ((int64_t)K_max_ctx + k) * nm, nm, t1) : 0;
                const int cell = TWO_ARM ? x0 * n1p + x1 : x0;
                const int r = rt[cell];
                const int rej = r < rho;
                r_acc += rej;
                x0_acc += rej ? x0 : 0;
                if (TWO_ARM) x1_acc += rej ? x1 : 0;
                if (SELECT) {
                    if (PACKED) atomicAdd(&hist[r >> 1], (r & 1) ? 0x10000u : 1u);
                    else atomicAdd(&hist[r], 1u);
                }
            }
        }
        // sixteen sims per thread and step: 16-byte loads of sixteen 8-bit counts;
        // full groups run without per-sim bounds tests, the last partial group with
        auto one_sim = [&](int x0, int x1) {
            const int cell = TWO_ARM ? x0 * n1p + x1 : x0;
            const int r = rt[cell];
            const int rej = r < rho;
            r_acc += rej;
            x0_acc += rej * x0;
            if (TWO_ARM) x1_acc += rej * x1;
            if (SELECT) {
                if (PACKED) atomicAdd(&hist[r >> 1], 1u << ((r & 1) << 4));
                else atomicAdd(&hist[r], 1u);
            }
        };
        int k16 = tid * 16;
        for (; !DIRECT && k16 + 16 <= Kc; k16 += NT * 16) {
            const uint4 w0 = *reinterpret_cast<const uint4*>(c0 + k16);
            const uint4 w1 = TWO_ARM ? *reinterpret_cast<const uint4*>(c1 + k16) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t a0[4] = {w0.x, w0.y, w0.z, w0.w};
            const uint32_t a1[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int j = 0; j < 16; ++j)
                one_sim((int)((a0[j >> 2] >> (8 * (j & 3))) & 0xFFu),
                        TWO_ARM ? (int)((a1[j >> 2] >> (8 * (j & 3))) & 0xFFu) : 0);
        }
        if (!DIRECT && k16 < Kc) {
            const uint4 w0 = *reinterpret_cast<const uint4*>(c0 + k16);
            const uint4 w1 = TWO_ARM ? *reinterpret_cast<const uint4*>(c1 + k16) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t a0[4] = {w0.x, w0.y, w0.z, w0.w};
            const uint32_t a1[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (k16 + j < Kc)
                    one_sim((int)((a0[j >> 2] >> (8 * (j & 3))) & 0xFFu),
                            TWO_ARM ? (int)((a1[j >> 2] >> (8 * (j & 3))) & 0xFFu) : 0);
        }
        r_acc = warp_sum(r_acc);
        x0_acc = warp_sum(x0_acc);
        if (TWO_ARM) x1_acc = warp_sum(x1_acc);
        if (lane == 0) {
            s_red[0][warp] = r_acc;
            s_red[1][warp] = x0_acc;
            s_red[2][warp] = x1_acc;
        }
        __syncthreads();
        double lam_i = -INFINITY;
        if (SELECT) {
            // k-th smallest rank: chunked prefix scan of the histogram (chunks of
            // whole words when packed)
            const int ks = badK ? 0 : o.ksel[i];
            int CH = (n_cells + NT - 1) / NT;
            if (PACKED) CH = (CH + 1) & ~1;
            const int b0 = min(tid * CH, n_cells), b1 = min(b0 + CH, n_cells);
            int local = 0;
            if (PACKED) {
                for (int w = b0 >> 1; w < (b1 + 1) >> 1; ++w) {
                    const uint32_t h = hist[w];
                    local += (int)(h & 0xFFFFu) + (int)(h >> 16);
                }
            } else {
                for (int b = b0; b < b1; ++b) local += (int)hist[b];
            }
            int incl = local;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            if (lane == 31) s_scan[warp] = incl;
            if (tid == 0) s_pick = -1;
            __syncthreads();
            int wpre = 0;
            for (int w = 0; w < warp; ++w) wpre += s_scan[w];
            incl += wpre;
            const int excl = incl - local;
            if (ks >= 1 && excl < ks && ks <= incl) {
                int cum = excl;
                for (int b = b0; b < b1; ++b) {
                    cum += bin_count<PACKED>(hist, b);
                    if (cum >= ks) {
                        s_pick = b;
                        break;
                    }
                }
            }
            __syncthreads();
            if (s_pick >= 0) lam_i = (double)vor_g[s_pick];
        }
        if (tid == 0) {
            if (badK) atomicOr(err, CSE_ERR_BAD_K);
            int64_t Rt = 0, X0 = 0, X1 = 0;
            for (int w = 0; w < (NT / 32); ++w) {
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
                const double s0 = badK ? NAN : o.sig[T.axis_off[0] + v0];
                o.score[i * d + 0] = (double)X0 - nm * s0 * (double)Rt;
                if (TWO_ARM) {
                    const double s1 = badK ? NAN : o.sig[T.axis_off[1] + v1];
                    o.score[i * d + 1] = (double)X1 - nm * s1 * (double)Rt;
                }
            }
            if (SELECT && o.lam_tile) o.lam_tile[i] = lam_i;
        }
        __syncthreads();
    }
}

// Statistic of every (tile, sim): S_out[off[i] + k] (testing and export).
__global__ void k_emit_ztest(TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride,
                             int32_t K_tiles, const float* __restrict__ S_g, int32_t n1p,
                             const int64_t* __restrict__ off, float* __restrict__ S_out, int32_t* __restrict__ err)
{
    const int last = D.n_looks - 1;
    for (int64_t i = blockIdx.x; i < T.n_tiles; i += gridDim.x) {
        const int K = T.K[i];
        const int v0 = T.center_idx[i * T.d];
        const int v1 = (T.d > 1) ? T.center_idx[i * T.d + 1] : 0;
        const bool bad = (K < 1) || (K > K_tiles) || v0 < 0 || v0 >= T.n_axis[0] ||
                         (T.d > 1 && (v1 < 0 || v1 >= T.n_axis[1]));
        if (bad) {
            if (threadIdx.x == 0) atomicOr(err, CSE_ERR_BAD_K);
            continue;
        }
        const uint8_t* c0 = cnt + ((int64_t)last * NA + T.axis_off[0] + v0) * k_stride;
        const uint8_t* c1 = (T.d > 1) ? cnt + ((int64_t)last * NA + T.axis_off[1] + v1) * k_stride : c0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const int cell = (T.d > 1) ? (int)c0[k] * n1p + (int)c1[k] : (int)c0[k];
            S_out[off[i] + k] = S_g[cell];
        }
    }
}

template <bool SEL, bool PACKED>
size_t smem_bytes(const cse_ctx* c)
{
    const size_t words = SEL ? (PACKED ? (size_t)(c->n_cells + 1) / 2 : (size_t)c->n_cells) : 0;
    return ((words + 3) & ~(size_t)3) * 4 + ((size_t)c->n_cells * 2 + 15) / 16 * 16;
}

// variant index: [direct][selection][packed][threads option]
inline int variant(bool direct, bool sel, bool packed, int topt)
{
    return (((direct ? 1 : 0) * 2 + (sel ? 1 : 0)) * 2 + (packed ? 1 : 0)) * 3 + topt;
}

template <bool TWO, bool SEL, bool PACKED, bool DIRECT, int NT>
int setup_one(cse_ctx* c, int topt)
{
    auto kern = k_sim_ztest<TWO, SEL, PACKED, DIRECT, NT>;
    const size_t smem = smem_bytes<SEL, PACKED>(c);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    c->sim_grid[variant(DIRECT, SEL, PACKED, topt)] = per_sm * c->num_sms;
    return CSE_OK;
}

template <bool TWO, bool SEL, bool PACKED, bool DIRECT, int NT>
int launch_one(cse_ctx* c, int topt, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
               double lambda, const SimOut& o, cudaStream_t s)
{
    int64_t grid = c->sim_grid[variant(DIRECT, SEL, PACKED, topt)];
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(c->counter, 0, sizeof(int32_t), s) != cudaSuccess) return CSE_CUDA_ERROR;
    cse_prof_begin(c, KID_SIM_ZTEST, s);
    k_sim_ztest<TWO, SEL, PACKED, DIRECT, NT><<<(unsigned)grid, NT, smem_bytes<SEL, PACKED>(c), s>>>(
        T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab, c->val_of_rank, c->n_cells, c->n1p,
        lambda_float_up(lambda), o, c->counter, c->err, c->U, c->thr, c->K_max);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

template <bool TWO, bool SEL, bool PACKED, bool DIRECT>
int setup_threads(cse_ctx* c)
{
    int st = setup_one<TWO, SEL, PACKED, DIRECT, 128>(c, 0);
    if (st == CSE_OK) st = setup_one<TWO, SEL, PACKED, DIRECT, 256>(c, 1);
    if (st == CSE_OK) st = setup_one<TWO, SEL, PACKED, DIRECT, 512>(c, 2);
    return st;
}

template <bool TWO, bool SEL, bool PACKED, bool DIRECT>
int launch_threads(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                   const SimOut& o, cudaStream_t s)
{
    switch (c->sim_topt) {
    case 0: return launch_one<TWO, SEL, PACKED, DIRECT, 128>(c, 0, T, NA, k_stride, K_tiles, lambda, o, s);
    case 2: return launch_one<TWO, SEL, PACKED, DIRECT, 512>(c, 2, T, NA, k_stride, K_tiles, lambda, o, s);
    default: return launch_one<TWO, SEL, PACKED, DIRECT, 256>(c, 1, T, NA, k_stride, K_tiles, lambda, o, s);
    }
}

template <bool TWO>
int setup_all(cse_ctx* c)
{
    int st = setup_threads<TWO, false, false, false>(c);
    if (st == CSE_OK) st = setup_threads<TWO, true, false, false>(c);
    if (st == CSE_OK) st = setup_threads<TWO, true, true, false>(c);
    if (st == CSE_OK) st = setup_threads<TWO, false, false, true>(c);
    if (st == CSE_OK) st = setup_threads<TWO, true, false, true>(c);
    if (st == CSE_OK) st = setup_threads<TWO, true, true, true>(c);
    return st;
}

template <bool TWO>
int launch_dispatch(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                    const SimOut& o, cudaStream_t s)
{
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    const bool packed = K_tiles < 65536;   // per-rank counts then fit 16 bits
    if (c->plain) {
        if (sel)
            return packed ? launch_threads<TWO, true, true, true>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                          : launch_threads<TWO, true, false, true>(c, T, NA, k_stride, K_tiles, lambda, o, s);
        return launch_threads<TWO, false, false, true>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
    if (sel) {
        return packed ? launch_threads<TWO, true, true, false>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                      : launch_threads<TWO, true, false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
    return launch_threads<TWO, false, false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
}

}  // namespace

int cse_launch_emit_ztest(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          const int64_t* off, float* S_out, cudaStream_t s)
{
    const int64_t grid = T.n_tiles < 4096 ? T.n_tiles : 4096;
    k_emit_ztest<<<(unsigned)grid, 256, 0, s>>>(T, c->D, c->cnt, NA, k_stride, K_tiles, c->S_tab, c->n1p, off, S_out,
                                                c->err);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_sim_ztest_setup(cse_ctx* c)
{
    if (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z) return setup_all<true>(c);
    return setup_all<false>(c);
}

int cse_launch_sim_ztest(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, int32_t k_stride, int32_t K_tiles,
                         double lambda, const SimOut& o, cudaStream_t s)
{
    if (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z)
        return launch_dispatch<true>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s);
    return launch_dispatch<false>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s);
}

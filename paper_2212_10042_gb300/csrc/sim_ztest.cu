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

constexpr int SIM_THREADS = 256;
constexpr int NWARP = SIM_THREADS / 32;

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool TWO_ARM, bool SELECT>
__global__ void __launch_bounds__(SIM_THREADS) k_sim_ztest(
    TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride, int32_t K_tiles,
    const uint16_t* __restrict__ rank_g, const float* __restrict__ S_g, const float* __restrict__ vor_g,
    int32_t n_cells, int32_t n1p, double lambda, SimOut o, int32_t* __restrict__ counter,
    int32_t* __restrict__ err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* hist = smem;                                               // [n_cells] if SELECT
    uint16_t* rt = reinterpret_cast<uint16_t*>(smem + (SELECT ? n_cells : 0));   // [n_cells]
    __shared__ int s_tile;
    __shared__ int s_rho;
    __shared__ int s_red[3][NWARP];
    __shared__ int s_scan[NWARP];
    __shared__ int s_pick;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_rho = 0;
    __syncthreads();
    int rho = 0;
    for (int c = tid; c < n_cells; c += SIM_THREADS) {
        rt[c] = rank_g[c];
        rho += ((double)S_g[c] < lambda) ? 1 : 0;
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
            for (int c = tid; c < n_cells; c += SIM_THREADS) hist[c] = 0u;
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
        // four sims per thread and step: 32-bit loads of four 8-bit counts
        for (int k4 = tid * 4; k4 < Kc; k4 += SIM_THREADS * 4) {
            const uint32_t w0 = *reinterpret_cast<const uint32_t*>(c0 + k4);
            const uint32_t w1 = TWO_ARM ? *reinterpret_cast<const uint32_t*>(c1 + k4) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k4 + j < Kc) {
                    const int x0 = (w0 >> (8 * j)) & 0xFF;
                    const int x1 = TWO_ARM ? ((w1 >> (8 * j)) & 0xFF) : 0;
                    const int cell = TWO_ARM ? x0 * n1p + x1 : x0;
                    const int r = rt[cell];
                    const int rej = r < rho;
                    r_acc += rej;
                    x0_acc += rej ? x0 : 0;
                    if (TWO_ARM) x1_acc += rej ? x1 : 0;
                    if (SELECT) atomicAdd(&hist[r], 1u);
                }
            }
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
            // k-th smallest rank: chunked prefix scan of the histogram
            const int ks = badK ? 0 : o.ksel[i];
            const int CH = (n_cells + SIM_THREADS - 1) / SIM_THREADS;
            const int b0 = tid * CH, b1 = min(b0 + CH, n_cells);
            int local = 0;
            for (int b = b0; b < b1; ++b) local += (int)hist[b];
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
                    cum += (int)hist[b];
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
            for (int w = 0; w < NWARP; ++w) {
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
                const double th0 = badK ? NAN : T.axis[0][v0];
                o.score[i * d + 0] = (double)X0 - nm / (1.0 + exp(-th0)) * (double)Rt;
                if (TWO_ARM) {
                    const double th1 = badK ? NAN : T.axis[1][v1];
                    o.score[i * d + 1] = (double)X1 - nm / (1.0 + exp(-th1)) * (double)Rt;
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

template <bool TWO, bool SEL>
size_t smem_bytes(const cse_ctx* c)
{
    return (SEL ? (size_t)c->n_cells * 4 : 0) + ((size_t)c->n_cells * 2 + 15) / 16 * 16;
}

template <bool TWO, bool SEL>
int setup_one(cse_ctx* c, int* grid)
{
    auto kern = k_sim_ztest<TWO, SEL>;
    const size_t smem = smem_bytes<TWO, SEL>(c);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SIM_THREADS, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    *grid = per_sm * c->num_sms;
    return CSE_OK;
}

template <bool TWO, bool SEL>
int launch_one(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
               const SimOut& o, cudaStream_t s)
{
    int64_t grid = c->sim_grid[SEL ? 1 : 0];
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(c->counter, 0, sizeof(int32_t), s) != cudaSuccess) return CSE_CUDA_ERROR;
    cse_prof_begin(c, KID_SIM_ZTEST, s);
    k_sim_ztest<TWO, SEL><<<(unsigned)grid, SIM_THREADS, smem_bytes<TWO, SEL>(c), s>>>(
        T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab, c->val_of_rank, c->n_cells, c->n1p,
        lambda, o, c->counter, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
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
    if (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z) {
        int st = setup_one<true, false>(c, &c->sim_grid[0]);
        return st != CSE_OK ? st : setup_one<true, true>(c, &c->sim_grid[1]);
    }
    int st = setup_one<false, false>(c, &c->sim_grid[0]);
    return st != CSE_OK ? st : setup_one<false, true>(c, &c->sim_grid[1]);
}

int cse_launch_sim_ztest(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, int32_t k_stride, int32_t K_tiles,
                         double lambda, const SimOut& o, cudaStream_t s)
{
    const bool two = (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z);
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    if (two) {
        return sel ? launch_one<true, true>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s)
                   : launch_one<true, false>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s);
    }
    return sel ? launch_one<false, true>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s)
               : launch_one<false, false>(c, T, n_axis_total, k_stride, K_tiles, lambda, o, s);
}

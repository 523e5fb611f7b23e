// sim_rand.cu -- the randomised z-tests (Sec. 7, after Thm. calibration): the
// statistic is the pair (S, w) with w the sim's independent tie-break word, the
// threshold the pair (lambda, c), compared lexicographically:
//   reject iff S < lambda, or S = lambda and w < c          (c = 0: S < lambda).
//
// Chosen form: the z-test cell-histogram pass (k_sim_cells) does the counting
// and the rank part of the selection, then k_tie handles what only the sims
// tying a threshold decide (below).  Plain form, also used when the cell
// histogram does not fit shared memory: k_sim_rand, one per-sim kernel.
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
    queue_reset(counter);
}

// Tie pass after the cell-histogram pass (k_sim_cells), the chosen form of the
// randomised test: one tile per CTA iteration.  The sims whose cell has rank r
// are those of the cells pos[r], ..., pos[r + ntie[r] - 1] (equal statistic;
// cells sorted by (S, index)); up to two of them are tested in registers, more
// through the rank table.
//  !SELECT (validation at (lambda, c)): the cell pass counted S < lambda into
//    o.R and o.Xrej; the sims of the cells tying lambda (rank rho, when lambda is
//    a table value and c > 0) whose word is below c are added, and the score is
//    formed from the totals.
//  SELECT (calibration): the cell pass left r*_i and m_i; the words of the sims
//    of rank r*_i are gathered into the CTA's buffer and the m_i-th smallest is
//    found by a radix select over four 8-bit digits: c_i.  The first kTieSmem
//    words are kept in shared memory, the rest in the CTA's global buffer.
constexpr int kTieSmem = 2048;

template <bool TWO_ARM, bool SELECT>
__global__ void __launch_bounds__(kRandThreads) k_tie(
    TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride, int32_t K_tiles,
    const uint16_t* __restrict__ rank_g, const float* __restrict__ S_g, const int32_t* __restrict__ pos_g,
    int32_t n_cells, int32_t n1p, double lambda, uint32_t c_thr, const uint32_t* __restrict__ W, SimOut o,
    uint32_t* __restrict__ c_tile, uint32_t* __restrict__ tbuf, int32_t* __restrict__ counter,
    int32_t* __restrict__ err)
{
    constexpr int NT = kRandThreads;
    constexpr int NW = NT / 32;
    __shared__ uint32_t hist[SELECT ? 256 : 1];
    __shared__ uint32_t sbuf[SELECT ? kTieSmem : 1];
    __shared__ int s_tile, s_next, s_rho, s_eq, s_g, s_ntc, s_tc[2];
    __shared__ int s_red[3][NW];
    __shared__ int s_scan[NW];
    __shared__ int s_res[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (SELECT)
        for (int b = tid; b < 256; b += NT) hist[b] = 0u;
    // validation: rank of the cells tying lambda (-1: lambda is not a table value, or c = 0)
    int tie_rank = -1;
    if (!SELECT) {
        if (tid == 0) {
            s_rho = 0;
            s_eq = 0;
        }
        __syncthreads();
        int rho = 0, eq = 0;
        for (int c = tid; c < n_cells; c += NT) {
            const double sv = (double)S_g[c];
            rho += (sv < lambda) ? 1 : 0;
            eq |= (sv == lambda) ? 1 : 0;
        }
        rho = rand_warp_sum(rho);
        eq = __any_sync(0xffffffffu, eq) ? 1 : 0;
        if (lane == 0) {
            atomicAdd(&s_rho, rho);
            if (eq) atomicOr(&s_eq, 1);
        }
        __syncthreads();
        tie_rank = (s_eq && c_thr > 0u) ? s_rho : -1;
    }
    const int last = D.n_looks - 1;
    const int d = T.d;
    uint32_t* buf = tbuf + (int64_t)blockIdx.x * K_tiles;
    if (tid == 0) s_next = atomicAdd(counter, 1);
    for (;;) {
        if (tid == 0) {
            s_tile = s_next;
            s_g = 0;
        }
        __syncthreads();
        const int64_t i = s_tile;
        if (i >= T.n_tiles) break;
        if (tid == 0) s_next = atomicAdd(counter, 1);   // the next tile, fetched while this one runs
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
        const int rs = SELECT ? (badK ? -1 : o.rstar[i]) : tie_rank;
        if (tid == 0) {   // the cells of rank rs
            int n = 0;
            if (rs >= 0 && rs < n_cells) {
                n = pos_g[n_cells + rs];
                s_tc[0] = pos_g[rs];
                s_tc[1] = (n > 1 && rs + 1 < n_cells) ? pos_g[rs + 1] : -1;
            }
            s_ntc = n;
        }
        __syncthreads();
        const int ntc = s_ntc;
        const int tc0 = ntc > 0 ? s_tc[0] : -1, tc1 = ntc > 1 ? s_tc[1] : -1;
        const bool by_rank = ntc > 2;
        // the tie cells' counts replicated into the four bytes of a word: a sim
        // of the four in a count word is in cell (a, b) iff its byte of
        // (q0 ^ rep(a)) | (q1 ^ rep(b)) is zero
        const uint32_t ra0 = (uint32_t)(TWO_ARM ? (tc0 >= 0 ? tc0 / n1p : 0) : (tc0 >= 0 ? tc0 : 0)) * 0x01010101u;
        const uint32_t rb0 = (uint32_t)(TWO_ARM && tc0 >= 0 ? tc0 % n1p : 0) * 0x01010101u;
        const uint32_t ra1 = (uint32_t)(TWO_ARM ? (tc1 >= 0 ? tc1 / n1p : 0) : (tc1 >= 0 ? tc1 : 0)) * 0x01010101u;
        const uint32_t rb1 = (uint32_t)(TWO_ARM && tc1 >= 0 ? tc1 % n1p : 0) * 0x01010101u;
        int r_acc = 0, x0_acc = 0, x1_acc = 0;
        if (ntc > 0) {
            // sixteen sims per thread and step from 16-byte loads of the count rows,
            // the next step's loads issued before this step's tests (k + 16 <= k_stride
            // for every 16-aligned k < Kc: k_stride is a multiple of 16)
            int k16 = tid * 16;
            uint4 n0 = make_uint4(0u, 0u, 0u, 0u), n1 = n0;
            if (k16 < Kc) {
                n0 = *reinterpret_cast<const uint4*>(c0 + k16);
                if (TWO_ARM) n1 = *reinterpret_cast<const uint4*>(c1 + k16);
            }
            for (; k16 < Kc; k16 += NT * 16) {
                const int kn = k16 + NT * 16;
                uint4 m0 = make_uint4(0u, 0u, 0u, 0u), m1 = m0;
                if (kn < Kc) {
                    m0 = *reinterpret_cast<const uint4*>(c0 + kn);
                    if (TWO_ARM) m1 = *reinterpret_cast<const uint4*>(c1 + kn);
                }
                const uint32_t q0[4] = {n0.x, n0.y, n0.z, n0.w};
                const uint32_t q1[4] = {n1.x, n1.y, n1.z, n1.w};
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    bool any = by_rank;
                    if (!by_rank) {
                        const uint32_t z0 = (q0[qq] ^ ra0) | (q1[qq] ^ rb0);
                        const uint32_t z1 = (q0[qq] ^ ra1) | (q1[qq] ^ rb1);
                        // a zero byte in z0 (or, with two tie cells, in z1)
                        uint32_t hz = (z0 - 0x01010101u) & ~z0;
                        if (ntc > 1) hz |= (z1 - 0x01010101u) & ~z1;
                        any = (hz & 0x80808080u) != 0u;
                    }
                    if (!any) continue;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int k = k16 + 4 * qq + b;
                        const int x0 = (int)((q0[qq] >> (8 * b)) & 0xFFu);
                        const int x1 = TWO_ARM ? (int)((q1[qq] >> (8 * b)) & 0xFFu) : 0;
                        const int cell = TWO_ARM ? x0 * n1p + x1 : x0;
                        const bool mem = by_rank ? ((int)__ldg(rank_g + min(cell, n_cells - 1)) == rs)
                                                 : (cell == tc0 || cell == tc1);
                        if (mem && k < Kc) {
                            const uint32_t wk = W[k];
                            if (SELECT) {
                                const int at = atomicAdd(&s_g, 1);
                                if (at < kTieSmem) sbuf[at] = wk;
                                else buf[at] = wk;
                            } else if (wk < c_thr) {
                                r_acc += 1;
                                x0_acc += x0;
                                x1_acc += x1;
                            }
                        }
                    }
                }
                n0 = m0;
                n1 = m1;
            }
        }
        if (SELECT) {
            __syncthreads();   // s_g final, the gathered words visible to the block
            uint32_t cval = 0u;
            if (rs >= 0) {     // block-uniform
                const int g = s_g;
                int m = o.mrem[i];   // 1 <= m <= g
                if (m < 1 || m > g) {   // cannot happen: the rank's sims hold m words
                    if (tid == 0) atomicOr(err, CSE_ERR_BAD_K);
                } else if (g <= NT) {
                    // one word a thread; its rank by (word, index); the thread of
                    // rank m - 1 holds the m-th smallest word
                    uint32_t v = 0u;
                    int rk = -1;
                    if (tid < g) {
                        v = sbuf[tid];
                        rk = 0;
                        for (int j = 0; j < g; ++j) {
                            const uint32_t u = sbuf[j];
                            rk += (u < v || (u == v && j < tid)) ? 1 : 0;
                        }
                    }
                    if (rk == m - 1) s_res[0] = (int)v;
                    __syncthreads();
                    cval = (uint32_t)s_res[0];
                } else {
                    uint32_t prefix = 0u, pmask = 0u;
                    for (int pass = 0; pass < 4; ++pass) {
                        const int sh = 24 - 8 * pass;
                        for (int k = tid; k < g; k += NT) {
                            const uint32_t v = (k < kTieSmem) ? sbuf[k] : buf[k];
                            if ((v & pmask) == prefix) atomicAdd(&hist[(v >> sh) & 0xFFu], 1u);
                        }
                        int bef = 0;
                        const int digit = block_find_kth<NT>(hist, 256, m, s_scan, s_res, &bef);
                        for (int b = tid; b < 256; b += NT) hist[b] = 0u;
                        __syncthreads();   // cleared before the next pass counts
                        if (digit < 0) {   // cannot happen: the rank's sims hold m words
                            if (tid == 0) atomicOr(err, CSE_ERR_BAD_K);
                            break;
                        }
                        m -= bef;
                        prefix |= (uint32_t)digit << sh;
                        pmask |= 0xFFu << sh;
                    }
                    cval = prefix;
                }
            }
            if (tid == 0) {
                if (badK) atomicOr(err, CSE_ERR_BAD_K);
                if (c_tile) c_tile[i] = cval;
            }
        } else {
            r_acc = rand_warp_sum(r_acc);
            x0_acc = rand_warp_sum(x0_acc);
            if (TWO_ARM) x1_acc = rand_warp_sum(x1_acc);
            if (lane == 0) {
                s_red[0][warp] = r_acc;
                s_red[1][warp] = x0_acc;
                s_red[2][warp] = x1_acc;
            }
            __syncthreads();
            if (tid == 0) {
                int64_t dR = 0, dX0 = 0, dX1 = 0;
                for (int w = 0; w < NW; ++w) {
                    dR += s_red[0][w];
                    dX0 += s_red[1][w];
                    dX1 += s_red[2][w];
                }
                const int64_t Rt = o.R[i] + dR;
                const int64_t X0 = o.Xrej[i * d + 0] + dX0;
                const int64_t X1 = TWO_ARM ? o.Xrej[i * d + 1] + dX1 : 0;
                o.R[i] = Rt;
                o.Xrej[i * d + 0] = X0;
                if (TWO_ARM) o.Xrej[i * d + 1] = X1;
                if (o.score) {
                    const double nm = (double)D.n_max;
                    const double s0 = badK ? NAN : o.sig[a0];
                    o.score[i * d + 0] = (double)X0 - nm * s0 * (double)Rt;
                    if (TWO_ARM) {
                        const double s1 = badK ? NAN : o.sig[a1];
                        o.score[i * d + 1] = (double)X1 - nm * s1 * (double)Rt;
                    }
                }
            }
        }
        __syncthreads();
    }
    queue_reset(counter);
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
        *key = ~0ull;   // reset for the next launch
        *ticket = 0u;
    }
}

template <bool TWO, bool SEL>
size_t rand_smem(const cse_ctx* c)
{
    const size_t hw = SEL ? (size_t)(c->n_cells > 2048 ? c->n_cells : 2048) : 0;
    return hw * 4 + ((size_t)c->n_cells * 2 + 15) / 16 * 16;
}

// Grows a device buffer to at least `bytes` (contents are not kept).
int grow_buf(void** p, size_t* cap, size_t bytes)
{
    if (bytes <= *cap && *p) return CSE_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, bytes < 256 ? 256 : bytes) != cudaSuccess) {
        cudaGetLastError();
        return CSE_OOM;
    }
    *cap = bytes < 256 ? 256 : bytes;
    return CSE_OK;
}

template <bool TWO, bool SEL>
int launch_tie(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
               uint32_t c_thr, const SimOut& o, uint32_t* c_tile, cudaStream_t s)
{
    auto kern = k_tie<TWO, SEL>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRandThreads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) grid = 1;
    if (SEL) {   // per-CTA buffer of tie-group words
        const int st = grow_buf((void**)&c->tbuf, &c->tbuf_cap, sizeof(uint32_t) * (size_t)grid * (size_t)K_tiles);
        if (st != CSE_OK) return st;
    }
    cse_prof_begin(c, KID_TIE, s);
    kern<<<(unsigned)grid, kRandThreads, 0, s>>>(T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab,
                                                c->cell_of_pos, c->n_cells, c->n1p, lambda, c_thr, c->tb, o, c_tile,
                                                c->tbuf, c->counter, c->err);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
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
    const bool two = c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z;
    if (!c->plain && c->cells_ok) {
        // chosen form: the cell-histogram pass, then the tie pass
        if (sel) {
            int st = grow_buf((void**)&c->tie_rm, &c->tie_cap, sizeof(int32_t) * 2 * (size_t)T.n_tiles);
            if (st != CSE_OK) return st;
            SimOut oc = o;
            oc.rstar = c->tie_rm;
            oc.mrem = c->tie_rm + T.n_tiles;
            st = cse_launch_sim_ztest(c, T, NA, k_stride, K_tiles, lambda, oc, s);
            if (st != CSE_OK) return st;
            return two ? launch_tie<true, true>(c, T, NA, k_stride, K_tiles, lambda, c_thr, oc, c_tile, s)
                       : launch_tie<false, true>(c, T, NA, k_stride, K_tiles, lambda, c_thr, oc, c_tile, s);
        }
        int64_t* R = o.R ? o.R : c->R;   // the context's scratch holds n_tiles (prepare_args)
        int64_t* X = o.Xrej;
        if (!X) {
            const int st = grow_buf((void**)&c->xs, &c->xs_cap, sizeof(int64_t) * (size_t)T.d * (size_t)T.n_tiles);
            if (st != CSE_OK) return st;
            X = c->xs;
        }
        SimOut oc = {o.sig, R, X, nullptr, nullptr, nullptr, nullptr, nullptr};
        const int st = cse_launch_sim_ztest(c, T, NA, k_stride, K_tiles, lambda, oc, s);
        if (st != CSE_OK) return st;
        oc.score = o.score;
        return two ? launch_tie<true, false>(c, T, NA, k_stride, K_tiles, lambda, c_thr, oc, nullptr, s)
                   : launch_tie<false, false>(c, T, NA, k_stride, K_tiles, lambda, c_thr, oc, nullptr, s);
    }
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
    // min_key is all ones and the ticket zero on entry (set at creation, restored by the last block)
    cse_prof_begin(c, KID_MIN, s);
    k_min_pair<<<(unsigned)blocks, 256, 0, s>>>(lam_tile, c_tile, n, lam_out, c_out, c->min_key, c->min_ticket);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

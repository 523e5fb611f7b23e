// sim_ztest.cu -- persistent simulation kernels for the one- and two-arm z-tests.
//
// For every tile i and sim k < K_i (Sec. 6.1 / 7.1): the success counts x_a are
// read from the axis count table (a binary search on the sorted CRN uniforms,
// done once per distinct axis value and sim), the design rejects iff the FP32
// statistic S(x) < lambda, and the tile accumulates
//   R = sum_k 1{rej},  Xrej_a = sum_k 1{rej} x_a            (exact integers),
//   score_a = Xrej_a - n_max sigmoid(theta_a) R              (FP64, Ex. exp-fam),
// and, with calibration on, the k_i-th smallest statistic (Eq.
// calibrated-threshold).
//
// k_sim_cells (the chosen path): each sim adds one to a shared-memory histogram
// over the count cells x = (x_0, x_1); R, Xrej and the order statistic are then
// read off the histogram once per tile, over the box of cells the tile's counts
// can reach (each axis value's least and greatest count, from a small kernel
// after the count table).  Every S(x) is a function of the cell, so this is the
// same sum regrouped by cell.  Ranks (the number of cells with a smaller statistic) order
// the cells: S(x) < lambda iff rank(x) < rho, rho = #{cells with S < lambda}.
//
// k_sim_direct (the plain comparison path): every (tile, sim, arm) count is its
// own binary search in the sorted uniforms, the statistic's rank is looked up
// per sim and a rank histogram is kept per sim.
//
// One CTA processes one tile at a time and pulls the next tile index from a
// global counter (persistent, load-balanced over uneven K_i).
#include <cuda_runtime.h>
#include <math.h>

#include "cse_internal.cuh"

namespace {

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
template <bool TWO_ARM, bool SELECT, bool PACKED, int NT>
__global__ void __launch_bounds__(NT) k_sim_direct(
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
        int r_acc = 0, x0_acc = 0, x1_acc = 0;
        {
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
    queue_reset(counter);
}

// Rank buckets of the order-statistic search in k_sim_cells: 64 ranks a bucket.
constexpr int kRankBucketBits = 6;
constexpr int kRankBucket = 1 << kRankBucketBits;

// Warp 0: the position of the ks-th unit in counts[0..n) (ks >= 1): returns the
// index b with sum(counts[0..b)) < ks <= sum(counts[0..b]) and the sum before it
// through *before, or -1; zeroes counts[0..n).  Called by all 32 lanes of warp 0.
__device__ __forceinline__ int warp_find_kth(uint32_t* counts, int n, int ks, int lane, int* before)
{
    const int per = (n + 31) / 32;
    const int b0 = min(lane * per, n), b1 = min(b0 + per, n);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += (int)counts[b];
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int excl = incl - local;
    int found = -1, fb = 0;
    if (ks >= 1 && excl < ks && ks <= incl) {
        int cum = excl;
        for (int b = b0; b < b1; ++b) {
            const int cb = (int)counts[b];
            if (cum + cb >= ks) {
                found = b;
                fb = cum;
                break;
            }
            cum += cb;
        }
    }
    for (int b = b0; b < b1; ++b) counts[b] = 0u;
    const unsigned who = __ballot_sync(0xffffffffu, found >= 0);
    if (who == 0u) return -1;
    const int src = __ffs(who) - 1;
    *before = __shfl_sync(0xffffffffu, fb, src);
    return __shfl_sync(0xffffffffu, found, src);
}

// One tile per CTA iteration.  Shared memory: the cell histogram over the
// tile's box [lo0, hi0] x [lo1, hi1] of reachable cells (the axis values' least
// and greatest counts), indexed j = (x0 - lo0) w + (x1 - lo1) with w = hi1 -
// lo1 + 1 and zero between tiles, box_cap cells; with selection, the
// rank-bucket counts.  Sized by the box instead of the whole count table
// (17 KB instead of 42 KB for n_max = 100), it leaves room for 9 CTAs of 128
// threads per SM instead of 5 of 256, and the tiles in flight hide the latency
// of each tile's loads, barriers and read-off.  The read-off splits the flat
// index j = row * w + col by an FP32 reciprocal (exact for j < 2^22); each
// thread keeps its first kCache populated cells in registers for the
// order-statistic pass.  A box of more than box_cap cells (only for far
// outlying counts) is histogrammed in slabs of whole rows, one pass over the
// tile's sims per slab (cells_slab_pass).
constexpr int kCache = 4;

// The slab form of the histogram for a box of more than box_cap cells: rows
// [r0, r0 + rps) at a time, one pass over the tile's sims per slab.  Phase 1
// (bsel < 0) returns this thread's sums of R, Xrej_0 and Xrej_1 over the
// rejecting cells and, with selection, adds the rank-bucket counts; phase 2
// adds the cells of rank bucket bsel into rcnt.  Every slab is zeroed after
// use.  Called by all TT threads of the tile's group (local index lt, group g).
template <int TT, int G>
__device__ __forceinline__ void group_sync(int g)
{
    // the TT threads of group g: named barrier 1 + g (barrier 0 is __syncthreads)
    if (G == 1) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(TT) : "memory");
}

template <bool TWO_ARM, int TT, int G>
__device__ __forceinline__ int3 cells_slab_pass(uint32_t* hist, uint32_t* bcnt, uint32_t* rcnt, const uint8_t* c0,
                                             const uint8_t* c1, int K, int lo0, int hi0, int lo1, int w, int rps,
                                             int n1p, int rho, bool sel, int bsel,
                                             const uint16_t* __restrict__ rank_g, int lt, int g)
{
    int3 acc = make_int3(0, 0, 0);
    for (int r0 = lo0; r0 <= hi0; r0 += rps) {
        const int r1 = min(hi0, r0 + rps - 1);
        for (int k = lt; k < K; k += TT) {
            const int x0 = (int)c0[k];
            if (x0 < r0 || x0 > r1) continue;
            const int col = TWO_ARM ? (int)c1[k] - lo1 : 0;
            atomicAdd(&hist[(x0 - r0) * w + col], 1u);
        }
        group_sync<TT, G>(g);
        const int ns = (r1 - r0 + 1) * w;
        for (int j = lt; j < ns; j += TT) {
            const uint32_t h = hist[j];
            if (h == 0u) continue;
            hist[j] = 0u;
            const int row = j / w, col = j - row * w;
            const int r = __ldg(rank_g + (r0 + row) * n1p + lo1 + col);
            if (bsel < 0) {
                if (r < rho) {
                    acc.x += (int)h;
                    acc.y += (int)h * (r0 + row);
                    acc.z += (int)h * (lo1 + col);
                }
                if (sel) atomicAdd(&bcnt[r >> kRankBucketBits], h);
            } else if ((r >> kRankBucketBits) == bsel) {
                atomicAdd(&rcnt[r & (kRankBucket - 1)], h);
            }
        }
        group_sync<TT, G>(g);
    }
    return acc;
}

// Tiles per CTA (G): the CTA's NT threads form G groups of TT = NT / G threads,
// each group working through its own tiles with its own histogram and rank
// counters, synchronised by its own named barrier.  More tiles in flight per
// SM for the same threads, barriers over fewer warps.
template <int NT>
constexpr int cells_min_blocks(int G)
{
    return NT == 64 ? 18 : (NT == 128 ? (G == 1 ? 9 : 8) : (NT == 256 ? 4 : 2));
}

template <bool TWO_ARM, bool SELECT, int NT, int G>
__global__ void __launch_bounds__(NT, cells_min_blocks<NT>(G)) k_sim_cells(
    TileArgs T, DesignArgs D, const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride, int32_t K_tiles,
    const uint16_t* __restrict__ rank_g, const float* __restrict__ S_g, const float* __restrict__ vor_g,
    int32_t n_cells, int32_t n1p, float lambda_up, SimOut o, int32_t* __restrict__ counter,
    int32_t* __restrict__ err, const uint32_t* __restrict__ bb, int32_t box_cap)
{
    pdl_entry();
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int TT = NT / G;      // threads of a tile
    constexpr int NW = TT / 32;     // warps of a tile
    static_assert(TT % 32 == 0 && TT >= 32, "a tile's group holds whole warps");
    const int n_buckets = (n_cells + kRankBucket - 1) >> kRankBucketBits;
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = tid / TT, lt = tid - g * TT, warp = lt >> 5;   // group, thread and warp in the group
    const int per_group = box_cap + (SELECT ? n_buckets + kRankBucket : 0);
    uint32_t* hist = smem + g * per_group;                                   // [box_cap]
    uint32_t* bcnt = hist + box_cap;                                         // [n_buckets]
    uint32_t* rcnt = bcnt + (SELECT ? n_buckets : 0);                        // [kRankBucket]
    __shared__ int s_tile[G];
    __shared__ int s_rho;
    __shared__ int s_red[G][3][NW];
    __shared__ int s_bsel[G], s_before[G], s_rank[G], s_mrem[G], s_next[G];
    __shared__ unsigned long long s_min[G];   // order key of the least lambda_i of the group's tiles

    if (tid == 0) s_rho = 0;
    if (tid < G) s_min[tid] = ~0ull;
    __syncthreads();
    int rho = 0;
    for (int c = tid; c < G * per_group; c += NT) smem[c] = 0u;
    for (int c = tid; c < n_cells; c += NT) rho += (S_g[c] < lambda_up) ? 1 : 0;
    rho = warp_sum(rho);
    if (lane == 0) atomicAdd(&s_rho, rho);
    __syncthreads();
    rho = s_rho;

    const int last = D.n_looks - 1;
    const int d = T.d;
    const int nm = D.n_max;
    if (lt == 0) s_next[g] = atomicAdd(counter, 1);
    for (;;) {
        if (lt == 0) s_tile[g] = s_next[g];
        group_sync<TT, G>(g);
        const int64_t i = s_tile[g];
        if (i >= T.n_tiles) break;
        if (lt == 0) s_next[g] = atomicAdd(counter, 1);   // the next tile, fetched while this one runs
        const int K = T.K[i];
        const int v0 = T.center_idx[i * d + 0];
        const int v1 = TWO_ARM ? T.center_idx[i * d + 1] : 0;
        // device-side argument checks: K_i in [1, K_max of the set], axis indices in range
        const bool badK = (K < 1) || (K > K_tiles) || v0 < 0 || v0 >= T.n_axis[0] ||
                          (TWO_ARM && (v1 < 0 || v1 >= T.n_axis[1]));
        const int Kc = badK ? 0 : K;
        const int a0 = T.axis_off[0] + (badK ? 0 : v0);
        const int a1 = TWO_ARM ? T.axis_off[1] + (badK ? 0 : v1) : 0;
        // per-tile inputs of the read-off and the epilogue, loaded before the sims
        const int ks = (SELECT && !badK) ? o.ksel[i] : 0;
        double sg0 = 0.0, sg1 = 0.0;
        if (lt == 0 && o.score) {
            sg0 = badK ? NAN : o.sig[a0];
            sg1 = (TWO_ARM && !badK) ? o.sig[a1] : NAN;
        }
        const uint8_t* c0 = cnt + ((int64_t)last * NA + a0) * k_stride;
        const uint8_t* c1 = TWO_ARM ? cnt + ((int64_t)last * NA + a1) * k_stride : c0;
        // the box of reachable cells (empty for a rejected tile), clamped to the table
        const int lo0 = badK ? 1 : (int)min(bb[a0], (uint32_t)nm);
        const int hi0 = badK ? 0 : (int)min(bb[NA + a0], (uint32_t)nm);
        const int lo1 = TWO_ARM ? (int)min(bb[a1], (uint32_t)nm) : 0;
        const int hi1 = TWO_ARM ? (int)min(bb[NA + a1], (uint32_t)nm) : 0;
        const int w = hi1 - lo1 + 1;
        const int nbox = (hi0 >= lo0 && w > 0) ? (hi0 - lo0 + 1) * w : 0;
        const bool slabs = nbox > box_cap;   // uniform over the group
        const int rps = max(1, box_cap / max(w, 1));
        const bool sel = SELECT && ks >= 1;
        int acc[3] = {0, 0, 0};   // R, Xrej_0, Xrej_1 over this thread's rejecting cells
        uint32_t c_rc[kCache], c_h[kCache];
#pragma unroll
        for (int t = 0; t < kCache; ++t) c_h[t] = 0u;
        const int base = lo0 * n1p + lo1;
        const float inv_w = 1.0f / (float)max(w, 1);

        if (!slabs) {
            // sixteen sims per thread and step from 16-byte loads of sixteen 8-bit
            // counts (the loads run two steps ahead of the increments)
            uint32_t* hb = hist - (TWO_ARM ? lo0 * w + lo1 : lo0);   // cell (x0, x1) at hb[x0 w + x1]
            const int Kf = nbox > 0 ? Kc : 0;
            int k16 = lt * 16;
            uint4 n0 = make_uint4(0u, 0u, 0u, 0u), n1 = n0, m0 = n0, m1 = n0;
            if (k16 + 16 <= Kf) {
                n0 = *reinterpret_cast<const uint4*>(c0 + k16);
                if (TWO_ARM) n1 = *reinterpret_cast<const uint4*>(c1 + k16);
            }
            if (k16 + TT * 16 + 16 <= Kf) {
                m0 = *reinterpret_cast<const uint4*>(c0 + k16 + TT * 16);
                if (TWO_ARM) m1 = *reinterpret_cast<const uint4*>(c1 + k16 + TT * 16);
            }
            for (; k16 + 16 <= Kf; k16 += TT * 16) {
                const uint32_t q0[4] = {n0.x, n0.y, n0.z, n0.w};
                const uint32_t q1[4] = {n1.x, n1.y, n1.z, n1.w};
                n0 = m0;
                n1 = m1;
                const int kn = k16 + 2 * TT * 16;
                if (kn + 16 <= Kf) {
                    m0 = *reinterpret_cast<const uint4*>(c0 + kn);
                    if (TWO_ARM) m1 = *reinterpret_cast<const uint4*>(c1 + kn);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int x0 = (int)((q0[j >> 2] >> (8 * (j & 3))) & 0xFFu);
                    const int cell = TWO_ARM ? x0 * w + (int)((q1[j >> 2] >> (8 * (j & 3))) & 0xFFu) : x0;
                    atomicAdd(&hb[cell], 1u);
                }
            }
            if (k16 < Kf) {
                const uint4 w0 = *reinterpret_cast<const uint4*>(c0 + k16);
                const uint4 w1 = TWO_ARM ? *reinterpret_cast<const uint4*>(c1 + k16) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t q0[4] = {w0.x, w0.y, w0.z, w0.w};
                const uint32_t q1[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (k16 + j < Kf) {
                        const int x0 = (int)((q0[j >> 2] >> (8 * (j & 3))) & 0xFFu);
                        const int cell = TWO_ARM ? x0 * w + (int)((q1[j >> 2] >> (8 * (j & 3))) & 0xFFu) : x0;
                        atomicAdd(&hb[cell], 1u);
                    }
                }
            }
            group_sync<TT, G>(g);

            // read-off: R, Xrej over the rejecting cells; with selection, counts per
            // rank bucket (the cells stay until the second pass)
            auto visit = [&](int j, bool cache, int t) {
                const int row = TWO_ARM ? __float2int_rz(((float)j + 0.5f) * inv_w) : j;
                const int col = TWO_ARM ? j - row * w : 0;
                const uint32_t h = hist[j];
                if (h == 0u) return;
                const int r = __ldg(rank_g + base + row * n1p + col);
                if (r < rho) {
                    acc[0] += (int)h;
                    acc[1] += (int)h * (lo0 + row);
                    acc[2] += (int)h * (lo1 + col);
                }
                if (sel) {
                    atomicAdd(&bcnt[r >> kRankBucketBits], h);
                    if (cache) {
                        c_rc[t] = (uint32_t)r;
                        c_h[t] = h;
                        hist[j] = 0u;
                    }
                } else {
                    hist[j] = 0u;
                }
            };
#pragma unroll
            for (int t = 0; t < kCache; ++t) {
                const int j = lt + t * TT;
                if (j < nbox) visit(j, true, t);
            }
            for (int j = lt + kCache * TT; j < nbox; j += TT) visit(j, false, 0);
        } else {
            const int3 a = cells_slab_pass<TWO_ARM, TT, G>(hist, bcnt, rcnt, c0, c1, Kc, lo0, hi0, lo1, w, rps, n1p,
                                                            rho, sel, -1, rank_g, lt, g);
            acc[0] = a.x;
            acc[1] = a.y;
            acc[2] = a.z;
        }
        int r_acc = warp_sum(acc[0]);
        int x0_acc = warp_sum(acc[1]);
        int x1_acc = TWO_ARM ? warp_sum(acc[2]) : 0;
        if (lane == 0) {
            s_red[g][0][warp] = r_acc;
            s_red[g][1][warp] = x0_acc;
            s_red[g][2][warp] = x1_acc;
        }
        double lam_i = -INFINITY;
        if (sel) {
            // the ks-th smallest statistic: its rank bucket, then its rank
            group_sync<TT, G>(g);
            if (warp == 0) {
                int before = 0;
                const int b = warp_find_kth(bcnt, n_buckets, ks, lane, &before);
                if (lane == 0) {
                    s_bsel[g] = b;
                    s_before[g] = before;
                }
            }
            group_sync<TT, G>(g);
            const int bsel = s_bsel[g];
            if (!slabs) {
#pragma unroll
                for (int t = 0; t < kCache; ++t) {
                    const int r = (int)c_rc[t];
                    if (c_h[t] != 0u && (r >> kRankBucketBits) == bsel)
                        atomicAdd(&rcnt[r & (kRankBucket - 1)], c_h[t]);
                }
                for (int j = lt + kCache * TT; j < nbox; j += TT) {
                    const uint32_t h = hist[j];
                    if (h == 0u) continue;
                    hist[j] = 0u;
                    const int row = TWO_ARM ? __float2int_rz(((float)j + 0.5f) * inv_w) : j;
                    const int col = TWO_ARM ? j - row * w : 0;
                    const int r = __ldg(rank_g + base + row * n1p + col);
                    if ((r >> kRankBucketBits) == bsel) atomicAdd(&rcnt[r & (kRankBucket - 1)], h);
                }
            } else if (bsel >= 0) {
                cells_slab_pass<TWO_ARM, TT, G>(hist, bcnt, rcnt, c0, c1, Kc, lo0, hi0, lo1, w, rps, n1p, rho, sel,
                                                bsel, rank_g, lt, g);
            }
            group_sync<TT, G>(g);
            if (warp == 0) {
                int before = 0;
                const int jr = (bsel >= 0) ? warp_find_kth(rcnt, kRankBucket, ks - s_before[g], lane, &before) : -1;
                if (lane == 0) {
                    s_rank[g] = (jr >= 0) ? (bsel << kRankBucketBits) + jr : -1;
                    s_mrem[g] = ks - s_before[g] - before;   // order of the ks-th sim among the rank's sims
                }
            }
            group_sync<TT, G>(g);
            if (s_rank[g] >= 0) lam_i = (double)vor_g[s_rank[g]];
        } else {
            group_sync<TT, G>(g);
        }
        if (o.cp_key && lt == (TT > 32 ? 32 : 0)) {   // the tile's (K, R) in the Clopper-Pearson memo,
            int64_t Rt = 0;   // as k_cp_mark would: a second warp, beside the epilogue of lt 0
            for (int w2 = 0; w2 < NW; ++w2) Rt += s_red[g][0][w2];
            o.cp_slot[i] = cp_memo_insert(((unsigned long long)(uint32_t)K << 32) | (uint32_t)Rt, o.cp_key, o.cp_cap,
                                          o.cp_list, o.cp_nkeys);
        }
        if (lt == 0) {
            if (badK) atomicOr(err, CSE_ERR_BAD_K);
            int64_t Rt = 0, X0 = 0, X1 = 0;
            for (int w2 = 0; w2 < NW; ++w2) {
                Rt += s_red[g][0][w2];
                X0 += s_red[g][1][w2];
                X1 += s_red[g][2][w2];
            }
            if (o.R) o.R[i] = Rt;
            if (o.Xrej) {
                o.Xrej[i * d + 0] = X0;
                if (TWO_ARM) o.Xrej[i * d + 1] = X1;
            }
            if (o.score) {
                const double nmd = (double)nm;
                o.score[i * d + 0] = (double)X0 - nmd * sg0 * (double)Rt;
                if (TWO_ARM) o.score[i * d + 1] = (double)X1 - nmd * sg1 * (double)Rt;
            }
            if (SELECT && o.lam_tile) o.lam_tile[i] = lam_i;
            if (SELECT) s_min[g] = min(s_min[g], order_key(lam_i));
            if (SELECT && o.rstar) {
                o.rstar[i] = sel ? s_rank[g] : -1;
                o.mrem[i] = sel ? s_mrem[g] : 0;
            }
        }
        group_sync<TT, G>(g);
    }
    __syncthreads();   // every group done before the queue is reset
    unsigned long long mine = ~0ull;
    if (tid == 0)
        for (int q = 0; q < G; ++q) mine = min(mine, s_min[q]);
    queue_reset_min(counter, o.min_key, mine, SELECT ? o.min_out : nullptr);
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
size_t direct_smem_bytes(const cse_ctx* c)
{
    const size_t words = SEL ? (PACKED ? (size_t)(c->n_cells + 1) / 2 : (size_t)c->n_cells) : 0;
    return ((words + 3) & ~(size_t)3) * 4 + ((size_t)c->n_cells * 2 + 15) / 16 * 16;
}

// Configurations of the cell-histogram kernel (threads per CTA, tiles per CTA),
// chosen by cse_autotune: index = c->cells_cfg.
constexpr int kCellsCfgs = 7;
constexpr int kCellsNT[kCellsCfgs] = {128, 256, 512, 64, 128, 256, 256};
constexpr int kCellsG[kCellsCfgs] = {1, 1, 1, 1, 2, 2, 4};

// cells of a tile's box histogram: the whole count table when it is smaller;
// 4,096 for a tile of 128 or more threads, 2,048 otherwise (more tiles per SM)
inline int cells_box_cap(const cse_ctx* c, int cfg)
{
    const int cap = (kCellsNT[cfg] / kCellsG[cfg] >= 128) ? CSE_CELLS_BOX : CSE_CELLS_BOX / 2;
    return c->n_cells < cap ? c->n_cells : cap;
}

template <bool SEL>
size_t cells_smem_bytes(const cse_ctx* c, int cfg)
{
    const size_t nb = SEL ? (size_t)((c->n_cells + kRankBucket - 1) >> kRankBucketBits) + kRankBucket : 0;
    return ((size_t)cells_box_cap(c, cfg) + nb) * 4 * kCellsG[cfg];
}

// variant index: [direct][selection][packed][threads option]
inline int variant(bool direct, bool sel, bool packed, int topt)
{
    return (((direct ? 1 : 0) * 2 + (sel ? 1 : 0)) * 2 + (packed ? 1 : 0)) * 3 + topt;
}

template <typename Kern>
int setup_kernel(cse_ctx* c, Kern kern, int nt, size_t smem, int var)
{
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    c->sim_grid[var] = per_sm * c->num_sms;
    return CSE_OK;
}

template <bool TWO, bool SEL, int CFG>
int setup_cells(cse_ctx* c)
{
    constexpr int NT = kCellsNT[CFG], G = kCellsG[CFG];
    auto kern = k_sim_cells<TWO, SEL, NT, G>;
    const size_t smem = cells_smem_bytes<SEL>(c, CFG);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return CSE_UNSUPPORTED_DESIGN;
    }
    c->cells_grid[SEL ? 1 : 0][CFG] = per_sm * c->num_sms;
    return CSE_OK;
}

template <bool TWO, bool SEL, bool PACKED, int NT>
int setup_direct(cse_ctx* c, int topt)
{
    return setup_kernel(c, k_sim_direct<TWO, SEL, PACKED, NT>, NT, direct_smem_bytes<SEL, PACKED>(c),
                        variant(true, SEL, PACKED, topt));
}

inline int64_t sim_grid(const cse_ctx* c, int var, int64_t n_tiles)
{
    int64_t grid = c->sim_grid[var];
    if (grid > n_tiles) grid = n_tiles;
    return grid < 1 ? 1 : grid;
}

template <bool TWO, bool SEL, int CFG>
int launch_cells(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                 const SimOut& o, cudaStream_t s)
{
    constexpr int NT = kCellsNT[CFG], G = kCellsG[CFG];
    int64_t grid = c->cells_grid[SEL ? 1 : 0][CFG];
    const int64_t need = (T.n_tiles + G - 1) / G;   // CTAs beyond this would find no tile
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    const int cap = cells_box_cap(c, CFG);
    const int box = (c->cells_box && c->cells_box < cap) ? c->cells_box : cap;
    if (SEL && o.min_out) c->min_folded = true;
    if (o.cp_key) c->cp_marked = true;
    cse_prof_begin(c, KID_SIM_ZTEST, s);
    cse_launch(c->pdl, k_sim_cells<TWO, SEL, NT, G>, dim3((unsigned)grid), dim3(NT), cells_smem_bytes<SEL>(c, CFG), s,
               T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab, c->val_of_rank, c->n_cells, c->n1p,
               lambda_float_up(lambda), o, c->counter, c->err, c->bb, box);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

template <bool TWO, bool SEL, bool PACKED, int NT>
int launch_direct(cse_ctx* c, int topt, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                  double lambda, const SimOut& o, cudaStream_t s)
{
    const int64_t grid = sim_grid(c, variant(true, SEL, PACKED, topt), T.n_tiles);
    cse_prof_begin(c, KID_SIM_ZTEST, s);
    k_sim_direct<TWO, SEL, PACKED, NT><<<(unsigned)grid, NT, direct_smem_bytes<SEL, PACKED>(c), s>>>(
        T, c->D, c->cnt, NA, k_stride, K_tiles, c->rank_tab, c->S_tab, c->val_of_rank, c->n_cells, c->n1p,
        lambda_float_up(lambda), o, c->counter, c->err, c->U, c->thr, c->K_max);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

template <bool TWO, bool SEL>
int setup_threads_cells(cse_ctx* c)
{
    int st = setup_cells<TWO, SEL, 0>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 1>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 2>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 3>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 4>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 5>(c);
    if (st == CSE_OK) st = setup_cells<TWO, SEL, 6>(c);
    return st;
}

template <bool TWO, bool SEL, bool PACKED>
int setup_threads_direct(cse_ctx* c)
{
    int st = setup_direct<TWO, SEL, PACKED, 128>(c, 0);
    if (st == CSE_OK) st = setup_direct<TWO, SEL, PACKED, 256>(c, 1);
    if (st == CSE_OK) st = setup_direct<TWO, SEL, PACKED, 512>(c, 2);
    return st;
}

template <bool TWO, bool SEL>
int launch_threads_cells(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                         double lambda, const SimOut& o, cudaStream_t s)
{
    switch (c->cells_cfg) {
    case 1: return launch_cells<TWO, SEL, 1>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    case 2: return launch_cells<TWO, SEL, 2>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    case 3: return launch_cells<TWO, SEL, 3>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    case 4: return launch_cells<TWO, SEL, 4>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    case 5: return launch_cells<TWO, SEL, 5>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    case 6: return launch_cells<TWO, SEL, 6>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    default: return launch_cells<TWO, SEL, 0>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
}

template <bool TWO, bool SEL, bool PACKED>
int launch_threads_direct(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          double lambda, const SimOut& o, cudaStream_t s)
{
    switch (c->sim_topt) {
    case 0: return launch_direct<TWO, SEL, PACKED, 128>(c, 0, T, NA, k_stride, K_tiles, lambda, o, s);
    case 2: return launch_direct<TWO, SEL, PACKED, 512>(c, 2, T, NA, k_stride, K_tiles, lambda, o, s);
    default: return launch_direct<TWO, SEL, PACKED, 256>(c, 1, T, NA, k_stride, K_tiles, lambda, o, s);
    }
}

template <bool TWO>
int setup_all(cse_ctx* c)
{
    // the cell histogram needs 4 bytes a cell of shared memory: larger designs
    // (two arms beyond n_max ~ 237) run the direct kernel only
    c->cells_ok = setup_threads_cells<TWO, false>(c) == CSE_OK && setup_threads_cells<TWO, true>(c) == CSE_OK;
    int st = setup_threads_direct<TWO, false, false>(c);
    if (st == CSE_OK) st = setup_threads_direct<TWO, true, false>(c);
    if (st == CSE_OK) st = setup_threads_direct<TWO, true, true>(c);
    return st;
}

template <bool TWO>
int launch_dispatch(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                    const SimOut& o, cudaStream_t s)
{
    const bool sel = (o.lam_tile != nullptr && o.ksel != nullptr);
    if (c->plain || !c->cells_ok) {
        const bool packed = K_tiles < 65536;   // per-rank counts then fit 16 bits
        if (sel)
            return packed ? launch_threads_direct<TWO, true, true>(c, T, NA, k_stride, K_tiles, lambda, o, s)
                          : launch_threads_direct<TWO, true, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
        return launch_threads_direct<TWO, false, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    }
    if (sel) return launch_threads_cells<TWO, true>(c, T, NA, k_stride, K_tiles, lambda, o, s);
    return launch_threads_cells<TWO, false>(c, T, NA, k_stride, K_tiles, lambda, o, s);
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

int cse_cells_configs() { return kCellsCfgs; }

void cse_cells_config(int cfg, int* threads, int* tiles)
{
    if (cfg < 0 || cfg >= kCellsCfgs) cfg = 0;
    if (threads) *threads = kCellsNT[cfg];
    if (tiles) *tiles = kCellsG[cfg];
}

int cse_cells_config_index(int threads, int tiles)
{
    for (int k = 0; k < kCellsCfgs; ++k)
        if (kCellsNT[k] == threads && kCellsG[k] == tiles) return k;
    return -1;
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

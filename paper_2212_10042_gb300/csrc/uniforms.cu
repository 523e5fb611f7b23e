// uniforms.cu -- common random numbers, success thresholds, axis count tables
// and statistic tables.
//
// CRN (Sec. 7.3 of the paper: simulations may be shared across tiles as long
// as each tile's own simulations are i.i.d.): sim k, arm a, patient j uses word
// j mod 4 of Philox4x32-10(counter (k, a, j/4, 0), key = seed).  The words of
// each (sim, arm) are sorted within every analysis segment
// [look_n[l-1], look_n[l]) so that the success count of any parameter value is
// a binary search (a patient succeeds iff u < t(theta)).
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "cse_internal.cuh"

namespace {

// One warp per (arm, sim) row: lane L generates and holds elements L*E .. L*E+E-1
// (E = 32-padded power of two / 32), and a bitonic network over the 32*E keys
// (in-register pairs when the partner distance is below E, warp shuffles above)
// sorts the row.  With several analysis segments the key carries the segment
// index above the word, so the row comes out sorted within each segment and
// segments in order; pad keys (all ones) sort last and are not written.
// Success threshold and sigmoid of axis value i of a tile set (flattened over
// the arms' axes).
__device__ __forceinline__ void threshold_of(int i, uint32_t* __restrict__ thr, double* __restrict__ sig,
                                             const TileArgs& T)
{
    int a = 0;
    while (a + 1 < T.d && i >= T.axis_off[a + 1]) ++a;
    const double th = T.axis[a][i - T.axis_off[a]];
    thr[i] = success_threshold(th);
    if (sig) sig[i] = 1.0 / (1.0 + exp(-th));
}

//
// Two small jobs ride on the first blocks (one thread each, before the rows):
// the randomised test's tie-break word of every sim (tb, may be NULL; word 0 of
// Philox4x32-10(counter (k, 0, 0, 1), key = seed), the patients' draws using
// counter word 3 = 0) and, when a tile set is given (thr not NULL), the success
// thresholds of its n_thr axis values: two launches fewer per step.
template <int E, bool SEG>
__global__ void __launch_bounds__(256) k_uniforms(uint32_t* __restrict__ U, int32_t K_max, int32_t d,
                                                  int32_t n_looks, int4 looks, int32_t n_max,
                                                  uint32_t key0, uint32_t key1, uint32_t* __restrict__ tb,
                                                  uint32_t* __restrict__ thr, double* __restrict__ sig, TileArgs T,
                                                  int32_t n_thr)
{
    pdl_entry();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tb && g < K_max) {
        u32x4 c = {(uint32_t)g, 0u, 0u, 1u};
        tb[g] = philox4x32_10(c, key0, key1).x;
    }
    if (thr && g < n_thr) threshold_of((int)g, thr, sig, T);
    using Key = typename std::conditional<SEG, unsigned long long, uint32_t>::type;
    constexpr int NP = 32 * E;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;   // row = a * K_max + k
    if (row >= (int64_t)d * K_max) return;                  // the whole warp leaves together
    const uint32_t a = (uint32_t)(row / K_max), k = (uint32_t)(row % K_max);
    Key v[E];
    u32x4 w = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int e = lane * E + i;
        if (i == 0 || (e & 3) == 0) {   // word j/4 of Philox(k, a, j/4, 0) holds element j
            u32x4 c = {k, a, (uint32_t)(e >> 2), 0u};
            w = philox4x32_10(c, key0, key1);
        }
        const uint32_t u = ((e & 3) == 0) ? w.x : ((e & 3) == 1) ? w.y : ((e & 3) == 2) ? w.z : w.w;
        if (SEG) {
            const unsigned long long seg = (unsigned long long)((n_looks > 1 && e >= looks.x) ? 1 : 0) +
                                           ((n_looks > 2 && e >= looks.y) ? 1 : 0);
            v[i] = (e < n_max) ? (Key)((seg << 32) | u) : (Key)~0ull;
        } else {
            v[i] = (e < n_max) ? (Key)u : (Key)0xFFFFFFFFu;
        }
    }
#pragma unroll
    for (int kk = 2; kk <= NP; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= E) {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int e = lane * E + i;
                    const Key p = __shfl_xor_sync(0xffffffffu, v[i], j / E);
                    const bool keep_min = ((e & kk) == 0) == ((e & j) == 0);
                    v[i] = keep_min ? (p < v[i] ? p : v[i]) : (p > v[i] ? p : v[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    if ((i & j) == 0) {
                        const int i2 = i | j;
                        const bool up = ((lane * E + i) & kk) == 0;
                        const Key x = v[i], y = v[i2];
                        const Key lo = x < y ? x : y, hi = x < y ? y : x;
                        v[i] = up ? lo : hi;
                        v[i2] = up ? hi : lo;
                    }
                }
            }
        }
    }
    uint32_t* out = U + row * n_max;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int e = lane * E + i;
        if (e < n_max) out[e] = (uint32_t)v[i];
    }
}

// Success threshold and sigmoid (for the score's grad A) of every axis value.
__global__ void k_thresholds(uint32_t* __restrict__ thr, double* __restrict__ sig, TileArgs T, int32_t n_total)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    threshold_of(i, thr, sig, T);
}

// Axis count table: cnt[(l * NA + off_a + v) * k_stride + k] = number of the
// first look_n[l] patients of (sim k, arm a) whose uniform is below t(axis_a[v]).
// Block: one arm, KB consecutive sims staged in shared memory (rows at an odd
// word stride, so that the 32 lanes' rows start in different banks).  Warp w
// takes a run of consecutive axis values for all KB sims (lane = sim): the
// thresholds of sorted axis values rise, so each look segment's count is a
// merge of the sorted uniforms with the thresholds (one binary search at the
// run's first value, then a forward scan: ~0.4 uniforms pass per axis step on
// the 256-value grids) instead of a binary search per value.  A threshold
// below the previous one (unsorted axis values) restarts with a binary search.
constexpr int KB = 32;
__global__ void __launch_bounds__(256) k_axis_counts(uint8_t* __restrict__ cnt, const uint32_t* __restrict__ U,
                                                     const uint32_t* __restrict__ thr, TileArgs T,
                                                     int32_t NA, int32_t K_max_ctx, int32_t K_tiles,
                                                     int32_t k_stride, int32_t n_looks, int4 looks,
                                                     int32_t n_max)
{
    pdl_entry();
    __shared__ uint32_t rows[KB * (CSE_MAX_NMAX + 1)];
    const int a = blockIdx.y;
    const int k0 = blockIdx.x * KB;
    const int nk = min(KB, K_tiles - k0);
    const int stride = n_max | 1;
    const uint32_t* src = U + ((int64_t)a * K_max_ctx + k0) * n_max;
    for (int i = threadIdx.x; i < nk * n_max; i += blockDim.x) {
        const int row = i / n_max;
        rows[row * stride + (i - row * n_max)] = src[i];
    }
    __syncthreads();
    const int kk = threadIdx.x & (KB - 1);
    const int nw = blockDim.x / KB, w = threadIdx.x / KB;
    // the arm's entries by selection (a runtime index into the by-value
    // argument would copy it to local memory)
    int na = T.n_axis[0], off = T.axis_off[0];
#pragma unroll
    for (int b = 1; b < CSE_MAX_ARMS; ++b)
        if (a == b) {
            na = T.n_axis[b];
            off = T.axis_off[b];
        }
    const int per = (na + nw - 1) / nw;
    const int v0 = w * per, v1 = min(v0 + per, na);
    if (kk >= nk || v0 >= v1) return;
    const uint32_t* r = rows + kk * stride;
    // look segments [0, L0), [L0, L1), [L1, L2) of the row (sorted within each)
    const int len0 = looks.x;
    const int len1 = (n_looks > 1) ? looks.y - looks.x : 0;
    const int len2 = (n_looks > 2) ? looks.z - looks.y : 0;
    const uint32_t* r1 = r + looks.x;
    const uint32_t* r2 = r + looks.y;
    uint32_t tp = thr[off + v0];
    int j0 = count_below(r, len0, tp), j1 = count_below(r1, len1, tp), j2 = count_below(r2, len2, tp);
    auto advance = [](const uint32_t* seg, int len, int jj, uint32_t t, bool back) {
        if (back) jj = count_below(seg, len, t);
        while (jj < len && seg[jj] < t) ++jj;
        return jj;
    };
    uint8_t* out = cnt + (int64_t)(off + v0) * k_stride + k0 + kk;
    const int64_t look_stride = (int64_t)NA * k_stride;
    for (int v = v0; v < v1; ++v, out += k_stride) {
        const uint32_t t = thr[off + v];
        const bool back = t < tp;
        tp = t;
        j0 = advance(r, len0, j0, t, back);
        out[0] = (uint8_t)j0;
        if (n_looks > 1) {
            j1 = advance(r1, len1, j1, t, back);
            out[look_stride] = (uint8_t)(j0 + j1);
            if (n_looks > 2) {
                j2 = advance(r2, len2, j2, t, back);
                out[2 * look_stride] = (uint8_t)(j0 + j1 + j2);
            }
        }
    }
}

// Least and greatest final-look count of each axis value over its first
// K_tiles sims: bb[v] and bb[NA + v].  One block per axis value, 16-byte loads
// folded with byte-wise min / max; the row's padding bytes past K_tiles (never
// written) are masked to the neutral values.
__global__ void __launch_bounds__(256) k_axis_box(const uint8_t* __restrict__ cnt, int32_t NA, int32_t k_stride,
                                                 int32_t K_tiles, int32_t last, uint32_t* __restrict__ bb)
{
    pdl_entry();
    const int v = blockIdx.x;
    const uint8_t* row = cnt + ((int64_t)last * NA + v) * k_stride;
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    for (int k16 = threadIdx.x * 16; k16 < K_tiles; k16 += blockDim.x * 16) {
        const uint4 w = *reinterpret_cast<const uint4*>(row + k16);
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            // bytes at or past K_tiles take the neutral values
            const int valid = min(max(K_tiles - (k16 + 4 * b), 0), 4);
            const uint32_t keep = valid >= 4 ? 0xFFFFFFFFu : ((1u << (8 * valid)) - 1u);
            lo = __vminu4(lo, q[b] | ~keep);
            hi = __vmaxu4(hi, q[b] & keep);
        }
    }
    // bytes to one value, then the block
    lo = min(min(lo & 0xFFu, (lo >> 8) & 0xFFu), min((lo >> 16) & 0xFFu, lo >> 24));
    hi = max(max(hi & 0xFFu, (hi >> 8) & 0xFFu), max((hi >> 16) & 0xFFu, hi >> 24));
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    __shared__ unsigned s_lo[8], s_hi[8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        bb[v] = lo;
        bb[NA + v] = hi;
    }
}

// FP32 statistics with correctly rounded operations in a fixed order (no FMA
// contraction: every step is an explicit __f*_rn intrinsic).
__device__ float stat_one_arm(int x, int n, double p0d)
{
    const float p0 = (float)p0d;
    const float fn = (float)n;
    const float num = __fsub_rn((float)x, __fmul_rn(fn, p0));
    float var = __fmul_rn(fn, p0);
    var = __fmul_rn(var, __fsub_rn(1.0f, p0));
    const float z = __fdiv_rn(num, __fsqrt_rn(var));
    return -z;
}

__device__ float stat_two_arm(int x0, int x1, int n0, int n1)
{
    const float fn0 = (float)n0, fn1 = (float)n1;
    const float p0 = __fdiv_rn((float)x0, fn0);
    const float p1 = __fdiv_rn((float)x1, fn1);
    const float pb = __fdiv_rn((float)(x0 + x1), __fadd_rn(fn0, fn1));
    const float inv = __fadd_rn(__fdiv_rn(1.0f, fn0), __fdiv_rn(1.0f, fn1));
    float var = __fmul_rn(pb, __fsub_rn(1.0f, pb));
    var = __fmul_rn(var, inv);
    float z = 0.0f;
    if (var > 0.0f) z = __fdiv_rn(__fsub_rn(p1, p0), __fsqrt_rn(var));
    return -z;
}

__global__ void k_stat_table(float* __restrict__ S, DesignArgs D, int32_t n_cells, int32_t n1p)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    if (D.stat == CSE_STAT_ONE_ARM_Z) {
        S[c] = stat_one_arm(c, D.n_max, D.p0);
    } else {
        S[c] = stat_two_arm(c / n1p, c % n1p, D.n_max, D.n_max);
    }
}

// rank[c] = #{c' : S[c'] < S[c]}; val_of_rank[rank[c]] = S[c] (equal S share a rank).
// With pos and ntie (may be NULL): pos[rank[c] + #{c' < c : S[c'] = S[c]}] = c,
// the cells sorted by (S, index), so the cells of rank r sit at positions r,
// r + 1, ..., r + ntie[r] - 1, ntie[r] = #{c' : S[c'] = S[c]}.
__global__ void k_rank_table(const float* __restrict__ S, uint16_t* __restrict__ rank,
                             float* __restrict__ vor, int32_t* __restrict__ pos, int32_t* __restrict__ ntie,
                             int32_t n_cells)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const float s = S[c];
    int r = 0, e = 0, t = 0;
    for (int j = 0; j < n_cells; ++j) {
        r += (S[j] < s);
        e += (j < c && S[j] == s);
        t += (S[j] == s);
    }
    rank[c] = (uint16_t)r;
    vor[r] = s;
    if (pos) {
        pos[r + e] = c;
        if (e == 0) ntie[r] = t;
    }
}

}  // namespace

int cse_launch_uniforms(cse_ctx* c, cudaStream_t s, const TileArgs* T, int32_t n_thr, bool* thr_done)
{
    const int64_t rows = (int64_t)c->D.d * c->K_max;
    const int blocks = (int)((rows + 7) / 8);
    int4 lk = make_int4(c->D.look_n[0], c->D.look_n[1], c->D.look_n[2], 0);
    const int n = c->D.n_max;
    const bool seg = c->D.n_looks > 1;
    const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
    // the side jobs need one thread each among the grid's blocks x 256 threads
    const bool fold = T != nullptr && n_thr > 0 && (int64_t)n_thr <= (int64_t)blocks * 256;
    TileArgs Tv;
    memset(&Tv, 0, sizeof(Tv));
    if (fold) Tv = *T;
    uint32_t* thr = fold ? c->thr : nullptr;
    double* sig = fold ? c->sig : nullptr;
    const int32_t nt = fold ? n_thr : 0;
    cse_prof_begin(c, KID_UNIFORMS, s);
#define CSE_UNIFORMS(E, SG)                                                                                       \
    cse_launch(c->pdl, k_uniforms<E, SG>, dim3(blocks), dim3(256), 0, s, c->U, c->K_max, c->D.d, c->D.n_looks, lk, \
               n, k0, k1, c->tb, thr, sig, Tv, nt)
    if (n <= 32) {
        if (seg) CSE_UNIFORMS(1, true);
        else CSE_UNIFORMS(1, false);
    } else if (n <= 64) {
        if (seg) CSE_UNIFORMS(2, true);
        else CSE_UNIFORMS(2, false);
    } else {
        if (seg) CSE_UNIFORMS(4, true);
        else CSE_UNIFORMS(4, false);
    }
#undef CSE_UNIFORMS
    cse_prof_end(c, s);
    c->launches += 1;
    if (thr_done) *thr_done = fold;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_tables(cse_ctx* c, cudaStream_t s)
{
    if (cse_posterior_design(c->D.stat)) return CSE_OK;
    const int n = c->n_cells;
    cse_prof_begin(c, KID_TABLES, s);
    k_stat_table<<<(n + 255) / 256, 256, 0, s>>>(c->S_tab, c->D, n, c->n1p);
    k_rank_table<<<(n + 255) / 256, 256, 0, s>>>(c->S_tab, c->rank_tab, c->val_of_rank, c->cell_of_pos,
                                                c->cell_of_pos ? c->cell_of_pos + n : nullptr, n);
    cse_prof_end(c, s);
    c->launches += 2;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_thresholds(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, cudaStream_t s)
{
    cse_prof_begin(c, KID_THRESHOLDS, s);
    cse_launch(c->pdl, k_thresholds, dim3((n_axis_total + 255) / 256), dim3(256), 0, s, c->thr, c->sig, T, n_axis_total);
    cse_prof_end(c, s);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_axis_counts(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, int32_t K_tiles,
                           int32_t k_stride, cudaStream_t s)
{
    dim3 grid((K_tiles + KB - 1) / KB, T.d);
    int4 lk = make_int4(c->D.look_n[0], c->D.look_n[1], c->D.look_n[2], 0);
    cse_prof_begin(c, KID_AXIS_COUNTS, s);
    cse_launch(c->pdl, k_axis_counts, dim3(grid), dim3(256), 0, s, c->cnt, c->U, c->thr, T, n_axis_total, c->K_max, K_tiles,
                                       k_stride, c->D.n_looks, lk, c->D.n_max);
    cse_launch(c->pdl, k_axis_box, dim3(n_axis_total), dim3(256), 0, s, c->cnt, n_axis_total, k_stride, K_tiles, c->D.n_looks - 1, c->bb);
    cse_prof_end(c, s);
    c->launches += 2;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

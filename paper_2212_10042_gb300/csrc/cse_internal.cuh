// cse_internal.cuh -- device helpers and the context layout of the CUDA path.
//
// GPU side only; nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/cse.h"

#define CSE_MAX_ARMS 4
#define CSE_MAX_LOOKS 3
#define CSE_MAX_NMAX 128
#define CSE_CELLS_BOX 4096   // cells a z-test tile's box histogram holds at once (16 KB)
#define CSE_MAX_KMAX (1 << 20)
#define CSE_BAYES_TABLE_MAX ((int64_t)1 << 27)   // entries of the tabulated posterior

// ---------------------------------------------------------------------------
// Philox4x32-10 in registers (Salmon et al., SC'11): two 32x32->64 products per
// round, high halves XORed with the round key into the other words; the key is
// advanced by the golden-ratio / sqrt(3) Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        u32x4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// floor(2^32 sigmoid(theta)) clamped to [0, 2^32 - 1], in FP64.
__device__ __forceinline__ uint32_t success_threshold(double theta)
{
    const double p = 1.0 / (1.0 + exp(-theta));
    const double y = p * 4294967296.0;
    if (!(y >= 0.0)) return 0u;
    if (y >= 4294967295.0) return 4294967295u;
    return (uint32_t)floor(y);
}

// Number of entries of the sorted array a[0..m) that are < t (lower bound).
__device__ __forceinline__ int count_below(const uint32_t* __restrict__ a, int m, uint32_t t)
{
    int base = 0;
    int len = m;
    while (len > 1) {
        const int half = len >> 1;
        base = (a[base + half] < t) ? base + half : base;
        len -= half;
    }
    return base + ((len == 1 && a[base] < t) ? 1 : 0);
}

// The smallest float >= lambda: for any float S, (double)S < lambda  <=>  S < it,
// so the rejection test runs in FP32 with the exact FP64 meaning (host side).
inline float lambda_float_up(double lambda)
{
    float f = (float)lambda;
    if ((double)f < lambda) f = nextafterf(f, INFINITY);
    return f;
}

// ---------------------------------------------------------------------------
// End of a persistent kernel's tile loop (every CTA calls it once, after its
// last draw from the queue): the last CTA to arrive resets the queue head
// counter[0] and the arrival ticket counter[1] to zero, so the next launch on
// the context starts from tile 0 without a memset.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void queue_reset(int32_t* counter)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {
            counter[0] = 0;
            counter[1] = 0;
        }
    }
}

// Order-preserving map of a double to uint64 (x < y iff key(x) < key(y); a NaN
// with the sign bit clear orders above +inf).
__device__ __forceinline__ unsigned long long order_key(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double order_unkey(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

// queue_reset with the minimum over tiles of the per-tile thresholds folded in
// (Eq. calibrated-threshold-final): every CTA's thread 0 adds its own minimum
// `mine` (an order key) to *min_key before taking its ticket, and the last CTA
// writes the decoded minimum to *min_out and sets *min_key back to all ones.
// Without min_out it is queue_reset.
__device__ __forceinline__ void queue_reset_min(int32_t* counter, unsigned long long* min_key,
                                                unsigned long long mine, double* min_out)
{
    if (threadIdx.x == 0) {
        if (min_out) atomicMin(min_key, mine);
        __threadfence();
        if (atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {
            if (min_out) {
                __threadfence();
                const unsigned long long k = atomicAdd(min_key, 0ull);
                *min_out = (k == ~0ull) ? INFINITY : order_unkey(k);
                *min_key = ~0ull;
            }
            counter[0] = 0;
            counter[1] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a step that cse_launch starts
// with programmatic stream serialization may be scheduled while the kernel
// before them in the stream is still running, which hides the launch latency
// between the short kernels of a step.  Each such kernel calls pdl_entry()
// before its first global memory access: griddepcontrol.wait returns once the
// previous grid has completed and its writes are visible (at once for a kernel
// launched without the attribute); launch_dependents then lets the next kernel
// in the stream be scheduled.  A kernel that waits before touching memory
// reads and writes exactly what it would in stream order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t cse_launch(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

// ---------------------------------------------------------------------------
// Hierarchical model of the Bayesian designs (Sec. 10.1): s2 integrated
// on kBayesNodes log-spaced nodes in [1e-6, 1e3], trapezoid in log s2.  Node j
// carries s2_j and the log of (trapezoid weight x InvGamma(0.0005, 0.000005)
// density at s2_j x Jacobian s2_j).
// ---------------------------------------------------------------------------
constexpr int kBayesNodes = 16;

struct NodeConst {
    float sig2[kBayesNodes];
    float lprior[kBayesNodes];
};

__device__ __forceinline__ NodeConst node_const()
{
    NodeConst C;
    const double lo = log(1e-6), hi = log(1e3);
    for (int j = 0; j < kBayesNodes; ++j) {
        const double L = lo + (hi - lo) * (double)j / (double)(kBayesNodes - 1);
        const double s2 = exp(L);
        const double trap = (j == 0 || j == kBayesNodes - 1) ? log(0.5) : 0.0;
        C.sig2[j] = (float)s2;
        C.lprior[j] = (float)(trap - (0.0005 + 1.0) * L - 0.000005 / s2 + L);
    }
    return C;
}

// ---------------------------------------------------------------------------
// Block-wide search of counts[0..n) for the position of the ks-th unit (ks >= 1):
// returns b with sum(counts[0..b)) < ks <= sum(counts[0..b]), and the sum before
// it in *before; -1 when the total is below ks.  All NT threads of the block call
// it; it ends with the result in every thread.  Uses s_scan[NT/32] and s_res[2] of
// the caller; the leading barrier keeps a previous call's readers of s_res ahead
// of the writes.
// ---------------------------------------------------------------------------
template <int NT>
__device__ int block_find_kth(const uint32_t* counts, int n, int ks, int* s_scan, int* s_res, int* before)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    const int per = (n + NT - 1) / NT;
    const int b0 = min(tid * per, n), b1 = min(b0 + per, n);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += (int)counts[b];
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
    if (ks >= 1 && excl < ks && ks <= incl) {
        int cum = excl;
        for (int b = b0; b < b1; ++b) {
            const int cb = (int)counts[b];
            if (cum + cb >= ks) {
                s_res[0] = b;
                s_res[1] = cum;
                break;
            }
            cum += cb;
        }
    }
    __syncthreads();
    *before = s_res[1];
    return s_res[0];
}

// ---------------------------------------------------------------------------
// Kernel argument bundles (passed by value).
// ---------------------------------------------------------------------------
struct TileArgs {
    int64_t n_tiles;
    int32_t d;
    int32_t n_axis[CSE_MAX_ARMS];
    int32_t axis_off[CSE_MAX_ARMS];  // offset of arm a in the flattened axis list
    const double* axis[CSE_MAX_ARMS];
    const int32_t* center_idx;
    const double* halfwidth;
    const uint32_t* null_mask;
    const int32_t* K;
};

struct DesignArgs {
    int32_t stat;
    int32_t d;
    int32_t n_looks;
    int32_t look_n[CSE_MAX_LOOKS];
    int32_t n_max;
    double p0;
    double drop;
    double tnull[CSE_MAX_ARMS];   // basket design: logit of each arm's null response rate
};

// the designs whose statistic is a tabulated posterior over count states
inline bool cse_posterior_design(int32_t stat)
{
    return stat == CSE_STAT_BAYES4 || stat == CSE_STAT_BERRY4;
}

// ---------------------------------------------------------------------------
// Kernel ids of the event profiler.
// ---------------------------------------------------------------------------
enum KernelId {
    KID_UNIFORMS = 0,
    KID_TABLES,
    KID_THRESHOLDS,
    KID_AXIS_COUNTS,
    KID_ALPHA_PRIME,
    KID_SIM_ZTEST,
    KID_SIM_BAYES4,
    KID_BAYES_TABLE,
    KID_BOUNDS,
    KID_CP,
    KID_MIN,
    KID_SIM_BASKET,
    KID_BASKET_TABLE,
    KID_TIE,
    KID_COUNT
};

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

// ---------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------
struct cse_ctx {
    DesignArgs D;
    uint64_t seed;
    int32_t K_max;
    int device;
    int64_t launches;
    // alpha' depends on the tiles alone: it runs on `side`, forked from and
    // joined back to the caller's stream by events, beside the table kernels
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;

    uint32_t* U;            // [d][K_max][n_max] uniforms sorted within each analysis segment
    uint32_t* tb;           // [K_max] tie-break word of each sim (randomised test)
    uint32_t* tbuf;         // [grid][K_max] tie-group words gathered by the randomised kernel
    size_t tbuf_cap;
    int64_t* xs;            // [n_tiles][d] success-sum scratch of the randomised validation
    size_t xs_cap;
    int32_t* tie_rm;        // [2][n_tiles] r* and m of the randomised calibration
    size_t tie_cap;
    float* S_tab;           // statistic table over count cells (z-tests)
    uint16_t* rank_tab;     // rank of each cell's S among all cells
    int32_t* cell_of_pos;   // [2][n_cells]: cells sorted by (S, cell index), the cells of rank r at
                            //   positions r ..; then the number of cells sharing rank r, at r
    float* val_of_rank;     // S value of each rank
    int32_t n_cells;        // cells of the table
    int32_t n1p;            // (n_max + 1): row length of the two-arm table

    // scratch grown on demand
    uint32_t* thr;          // [sum n_axis] success thresholds of the axis values
    size_t thr_cap;
    double* sig;            // [sum n_axis] sigmoid of the axis values (grad A / n_max)
    size_t sig_cap;
    uint8_t* cnt;           // axis count table [look][axis value][K stride]
    size_t cnt_cap;
    uint32_t* bb;           // [2][n_axis_total] least / greatest final-look success count over
    size_t bb_cap;          //   the simulations of each axis value: the box of cells a tile reaches
    int32_t* ksel;          // [n_tiles] order-statistic index (calibration)
    double* aprime;         // [n_tiles] alpha' scratch
    double* lam_tile;       // [n_tiles] per-tile lambda scratch
    int64_t* R;             // [n_tiles] reject count scratch
    size_t tile_cap;
    unsigned long long* cp_key;   // hash table of distinct (K, R) pairs (power-of-two capacity)
    double* cp_val;         // Clopper-Pearson bound of each occupied slot
    int32_t* cp_slot;       // [n_tiles] slot of each tile's (K, R)
    uint32_t* cp_list;      // [n_tiles] occupied slots, in insertion order
    int32_t* cp_nkeys;      // number of occupied slots
    uint64_t cp_cap;
    int32_t* counter;       // work-queue head of the persistent kernels
    unsigned long long* min_key;   // order key of the running minimum (k_min)
    unsigned int* min_ticket;      // blocks of k_min finished (zero between launches)
    double* geom;           // [n_tiles][d][3] per-arm softplus terms from alpha' (cse_step)
    size_t geom_cap;
    int32_t* err;           // device-side check / timeout flags
    double* lam_dev;        // global lambda scratch
    double* lam_host;       // pinned host scalar
    int32_t num_sms;
    int32_t sim_grid[24];   // persistent grid of the simulation kernel [direct][selection][packed][threads]
    int32_t sim_topt;       // threads option of the per-sim simulation kernels (0: 128, 1: 256, 2: 512)
    int32_t cells_cfg;      // (threads, tiles) per CTA of the z-test cell kernel (sim_ztest.cu), 0: (128, 1)
    int32_t cells_grid[2][8];   // its persistent grid per [selection][configuration]
    bool cells_ok;          // the cell-histogram kernel fits this design's shared memory
    int32_t cells_box;      // box capacity of the cell histogram in cells (0: the allocated one)
    bool pdl;               // step kernels start with programmatic dependent launch
    bool min_folded;        // the last simulation launch wrote the minimum over tiles (SimOut::min_out)
    bool cp_marked;         // the last simulation launch filled the Clopper-Pearson memo (SimOut::cp_key)

    bool plain;             // plain comparison path: direct counts, FP64-only bounds
    bool u_stale;           // cse_reseed changed the key; U and tb not yet regenerated

    // four-arm Bayesian design: tabulated posterior (see sim_bayes4.cu)
    bool bt_tables;         // tables built
    bool bt_direct;         // evaluate the posterior per simulation instead
    uint8_t* bt_d1;         // drop bits at the first analysis
    uint8_t* bt_d2;         // drop bits at the second analysis
    uint32_t* bt_d2s;       // the same over sorted code triples, 3 bits an entry (packed form)
    bool bt_packed;         // the simulation kernel runs the packed per-trial form
    float4* bt_f4;          // final-analysis P(theta_self > theta_0) of the three treatments per sorted code triple
    float4* bk_q;           // basket design: (1 - P(theta_i > t_i | x)) per count state (see sim_basket.cu)
    uint32_t* keys;         // per-CTA statistic keys for order-statistic selection
    size_t keys_cap;

    // simulation at arbitrary points (cse_type1_error): the axis-indexed form
    // built on the device (see points.cu)
    unsigned long long* pt_keys;   // [d][pt_P] hash keys: the coordinates' bits
    int32_t* pt_vals;       // [d][pt_P] dense index of each occupied slot
    int32_t* pt_count;      // [4] distinct coordinates per arm (device)
    int32_t* pt_count_host; // [4] the same, read back (pinned host)
    double* pt_axis;        // [d][pt_cap] distinct coordinates of each arm
    int32_t* pt_idx;        // [pt_cap][d] each point's index into its arms' coordinates
    uint32_t pt_P;          // hash capacity per arm (a power of two > pt_cap)
    size_t pt_cap;          // points the scratch holds

    // event profiler
    bool prof_on;
    int prof_only = -1;       // kernel id timed alone, or -1 for all
    bool prof_skip = false;   // the last cse_prof_begin recorded nothing
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    double prof_ms[KID_COUNT];
    int64_t prof_n[KID_COUNT];
};

// bracket a kernel launch with profiler events (no-ops unless enabled)
void cse_prof_begin(cse_ctx* c, int kid, cudaStream_t s);
void cse_prof_end(cse_ctx* c, cudaStream_t s);

// error flag bits written by kernels
#define CSE_ERR_BAD_K 1
#define CSE_ERR_TIMEOUT 2

// ---------------------------------------------------------------------------
// Launchers implemented in the .cu files (host functions).
// ---------------------------------------------------------------------------
// With a tile set T (else NULL), the uniforms kernel's first blocks also write
// the success thresholds of its n_thr axis values; *thr_done says whether they did.
int cse_launch_uniforms(cse_ctx* c, cudaStream_t s, const TileArgs* T = nullptr, int32_t n_thr = 0,
                        bool* thr_done = nullptr);
int cse_launch_tables(cse_ctx* c, cudaStream_t s);
int cse_launch_thresholds(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, cudaStream_t s);
int cse_launch_axis_counts(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, int32_t K_tiles,
                           int32_t k_stride, cudaStream_t s);
int cse_bound_set_attrs();   // once per context: launch attributes of the bound kernels
int cse_launch_alpha_prime(cse_ctx* c, const TileArgs& T, double alpha, double* aprime_out, int32_t* ksel,
                           cudaStream_t s, double* geom = nullptr);

// Clopper-Pearson memo (bound.cu): the distinct (K, R) keys of a call in an
// open-addressing table (linear probing over at most cap slots, cap a power of
// two, no waiting), each first insertion listed for the solve.  Key: a tag bit
// (63), K (bits 32..62), R.  Returns the key's slot, -1 if the table is full.
constexpr unsigned long long kCpEmptyKey = ~0ull;

__device__ __forceinline__ int32_t cp_memo_insert(unsigned long long key, unsigned long long* keys, uint32_t cap,
                                                  uint32_t* list, int32_t* n_keys)
{
    unsigned long long hk = key;   // fmix64 finaliser, first half
    hk ^= hk >> 33;
    hk *= 0xff51afd7ed558ccdull;
    hk ^= hk >> 33;
    uint32_t h = (uint32_t)hk & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const unsigned long long old = atomicCAS(&keys[h], kCpEmptyKey, key);
        if (old == kCpEmptyKey) list[atomicAdd(n_keys, 1)] = h;   // first insertion: list the key
        if (old == kCpEmptyKey || old == key) return (int32_t)h;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

struct SimOut {
    const double* sig;   // sigmoid of each axis value (flattened like the thresholds)
    int64_t* R;
    int64_t* Xrej;
    double* score;
    double* lam_tile;   // calibration output (requires ksel)
    const int32_t* ksel;
    int32_t* rstar;     // z-test cell kernel, calibration: rank of lambda_i's cells (-1: k_i = 0)
    int32_t* mrem;      //   and the order of the k_i-th sim within that rank's sims
    // calibration: min over tiles of lambda_i written to *min_out (device) by the
    // kernel's last CTA, through *min_key (all ones between launches); kernels
    // that do so set the context's min_folded
    unsigned long long* min_key;
    double* min_out;
    // upper Clopper-Pearson memo (set by cse_step): kernels that take it insert
    // each tile's (K, R) key and its slot themselves and set the context's
    // cp_marked, so that the bound pass needs no k_cp_mark
    unsigned long long* cp_key;
    uint32_t cp_cap;
    int32_t* cp_slot;
    uint32_t* cp_list;
    int32_t* cp_nkeys;
};
int cse_sim_ztest_setup(cse_ctx* c);
// configurations (threads per block, tiles per block) of the z-test cell kernel
int cse_cells_configs();
void cse_cells_config(int cfg, int* threads, int* tiles);
int cse_cells_config_index(int threads, int tiles);   // -1 if not built
int cse_launch_sim_ztest(cse_ctx* c, const TileArgs& T, int32_t n_axis_total, int32_t k_stride,
                         int32_t K_tiles, double lambda, const SimOut& o, cudaStream_t s);
int cse_bayes4_setup(cse_ctx* c, cudaStream_t s);
int cse_launch_emit_ztest(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          const int64_t* off, float* S_out, cudaStream_t s);
int cse_launch_emit_bayes4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                           const int64_t* off, float* S_out, cudaStream_t s);
int cse_launch_sim_bayes4(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          double lambda, const SimOut& o, cudaStream_t s);
int cse_basket_setup(cse_ctx* c, cudaStream_t s);
int cse_launch_sim_basket(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                          double lambda, const SimOut& o, cudaStream_t s);
int cse_launch_emit_basket(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles,
                           const int64_t* off, float* S_out, cudaStream_t s);
// marked: the simulation kernel already filled the upper Clopper-Pearson memo
int cse_launch_bounds(cse_ctx* c, const TileArgs& T, const int64_t* R, double delta, bool lower, double* u0,
                      double* bound, double* qstar, cudaStream_t s, const double* geom = nullptr,
                      bool marked = false);
int cse_launch_sim_rand(cse_ctx* c, const TileArgs& T, int32_t NA, int32_t k_stride, int32_t K_tiles, double lambda,
                        uint32_t c_thr, const SimOut& o, uint32_t* c_tile, cudaStream_t s);
int cse_launch_min_pair(cse_ctx* c, const double* lam_tile, const uint32_t* c_tile, int64_t n, double* lam_out,
                        uint32_t* c_out, cudaStream_t s);
int cse_launch_min(cse_ctx* c, const double* lam_tile, int64_t n, double* out, cudaStream_t s);
int cse_launch_backward(int64_t n, int32_t d, const double* g, const double* score, const int32_t* K,
                        double* out, cudaStream_t s);
int cse_launch_point_axes(cse_ctx* c, const double* theta, int64_t n, int32_t d, cudaStream_t s);
int cse_launch_fhat(cse_ctx* c, const int64_t* R, const int32_t* K, int64_t n, double* fhat, cudaStream_t s);

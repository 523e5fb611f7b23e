// capi.cu -- the C ABI (include/cse.h): context lifetime, argument checks,
// scratch management and the order of the kernels of each call.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "cse_internal.cuh"

#define CSE_TRY(expr)                       \
    do {                                    \
        int _st = (expr);                   \
        if (_st != CSE_OK) return _st;      \
    } while (0)

#define CUDA_TRY(expr)                                  \
    do {                                                \
        if ((expr) != cudaSuccess) {                    \
            cudaGetLastError();                         \
            return CSE_CUDA_ERROR;                      \
        }                                               \
    } while (0)

static const char* const kKernelNames[KID_COUNT] = {
    "uniforms", "stat_tables", "thresholds", "axis_counts", "alpha_prime",
    "sim_ztest", "sim_bayes4", "bayes_table", "bounds", "cp_distinct", "min_lambda",
    "sim_basket", "basket_table", "tie_pass"};

namespace {

cudaEvent_t prof_event(cse_ctx* c)
{
    if (!c->prof_free.empty()) {
        cudaEvent_t e = c->prof_free.back();
        c->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int grow(void** p, size_t* cap, size_t bytes)
{
    if (bytes <= *cap && *p) return CSE_OK;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(p, want) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return CSE_OOM;
    }
    *cap = want;
    return CSE_OK;
}

struct Prepared {
    TileArgs T;
    int32_t NA;
    int32_t K_tiles;
    int32_t k_stride;
};

// geom: the call reads the tiles' half-widths (bounds, alpha'); the
// simulation alone does not
int prepare_args(cse_ctx* c, const cse_tiles* t, Prepared* P, bool geom = true)
{
    if (!c || !t) return CSE_INVALID_ARG;
    if (t->n_tiles < 1 || !t->center_idx || (geom && !t->halfwidth) || !t->null_mask || !t->K) return CSE_INVALID_ARG;
    if (t->K_max < 1 || t->K_max > c->K_max) return CSE_INVALID_ARG;
    const int d = c->D.d;
    TileArgs& T = P->T;
    memset(&T, 0, sizeof(T));
    T.n_tiles = t->n_tiles;
    T.d = d;
    int32_t na = 0;
    for (int a = 0; a < d; ++a) {
        if (t->n_axis[a] < 1 || !t->axis[a]) return CSE_INVALID_ARG;
        T.n_axis[a] = t->n_axis[a];
        T.axis_off[a] = na;
        T.axis[a] = t->axis[a];
        na += t->n_axis[a];
    }
    T.center_idx = t->center_idx;
    T.halfwidth = t->halfwidth;
    T.null_mask = t->null_mask;
    T.K = t->K;
    P->NA = na;
    P->K_tiles = t->K_max;
    P->k_stride = (t->K_max + 15) / 16 * 16;

    CSE_TRY(grow((void**)&c->thr, &c->thr_cap, sizeof(uint32_t) * (size_t)na));
    CSE_TRY(grow((void**)&c->sig, &c->sig_cap, sizeof(double) * (size_t)na));
    const size_t cnt_bytes = (size_t)c->D.n_looks * (size_t)na * (size_t)P->k_stride;
    CSE_TRY(grow((void**)&c->cnt, &c->cnt_cap, cnt_bytes));
    CSE_TRY(grow((void**)&c->bb, &c->bb_cap, sizeof(uint32_t) * 2 * (size_t)na));
    if ((size_t)t->n_tiles > c->tile_cap) {
        cudaFree(c->ksel);
        cudaFree(c->aprime);
        cudaFree(c->lam_tile);
        cudaFree(c->R);
        c->ksel = nullptr;
        c->aprime = c->lam_tile = nullptr;
        c->R = nullptr;
        c->tile_cap = 0;
        const size_t n = (size_t)t->n_tiles;
        if (cudaMalloc(&c->ksel, n * 4) != cudaSuccess || cudaMalloc(&c->aprime, n * 8) != cudaSuccess ||
            cudaMalloc(&c->lam_tile, n * 8) != cudaSuccess || cudaMalloc(&c->R, n * 8) != cudaSuccess) {
            cudaGetLastError();
            return CSE_OOM;
        }
        c->tile_cap = n;
    }
    if (c->cp_cap < 2 * (uint64_t)t->n_tiles) {
        uint64_t cap = 1024;
        while (cap < 2 * (uint64_t)t->n_tiles) cap <<= 1;
        cudaFree(c->cp_key);
        cudaFree(c->cp_val);
        cudaFree(c->cp_slot);
        cudaFree(c->cp_list);
        c->cp_key = nullptr;
        c->cp_val = nullptr;
        c->cp_slot = nullptr;
        c->cp_list = nullptr;
        c->cp_cap = 0;
        if (cap > 0xFFFFFFFFull ||
            cudaMalloc(&c->cp_key, sizeof(unsigned long long) * cap) != cudaSuccess ||
            cudaMalloc(&c->cp_val, sizeof(double) * cap) != cudaSuccess ||
            cudaMalloc(&c->cp_slot, sizeof(int32_t) * (size_t)t->n_tiles * 2) != cudaSuccess ||
            cudaMalloc(&c->cp_list, sizeof(uint32_t) * (size_t)t->n_tiles * 2) != cudaSuccess) {
            cudaGetLastError();
            return CSE_OOM;
        }
        // an empty key table (the solve empties it again after each use)
        if (cudaMemset(c->cp_key, 0xFF, sizeof(unsigned long long) * cap) != cudaSuccess) {
            cudaGetLastError();
            return CSE_CUDA_ERROR;
        }
        c->cp_cap = cap;
    }
    return CSE_OK;
}

// Uniforms of a new key if pending, success thresholds of every axis
// coordinate, then the axis count tables.
int launch_tables(cse_ctx* c, const Prepared& P, cudaStream_t s)
{
    bool thr_done = false;   // a new key's uniforms kernel writes the thresholds as well
    if (c->u_stale) {
        CSE_TRY(cse_launch_uniforms(c, s, &P.T, P.NA, &thr_done));
        c->u_stale = false;
    }
    if (!thr_done) CSE_TRY(cse_launch_thresholds(c, P.T, P.NA, s));
    // the plain z-test path searches the sorted uniforms per (tile, sim) instead
    if (!(c->plain && !cse_posterior_design(c->D.stat)))
        CSE_TRY(cse_launch_axis_counts(c, P.T, P.NA, P.K_tiles, P.k_stride, s));
    return CSE_OK;
}

int prepare(cse_ctx* c, const cse_tiles* t, cudaStream_t s, Prepared* P, bool geom = true)
{
    CSE_TRY(prepare_args(c, t, P, geom));
    return launch_tables(c, *P, s);
}

// alpha' (and the order-statistic index of each tile) on the side stream, in
// parallel with the table kernels (and the uniforms of a new key); the caller's
// stream waits for it before the simulation pass reads ksel.  Capturable into a
// CUDA graph (event fork/join).
int tables_and_alpha_prime(cse_ctx* c, const Prepared& P, double alpha, double* aprime_out, cudaStream_t s,
                           double* geom = nullptr)
{
    CUDA_TRY(cudaEventRecord(c->ev_fork, s));
    CUDA_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    CSE_TRY(cse_launch_alpha_prime(c, P.T, alpha, aprime_out, c->ksel, c->side, geom));
    CUDA_TRY(cudaEventRecord(c->ev_join, c->side));
    CSE_TRY(launch_tables(c, P, s));
    CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
    return CSE_OK;
}

int sim_pass(cse_ctx* c, const Prepared& P, double lambda, const SimOut& o, cudaStream_t s)
{
    c->min_folded = false;   // set by a kernel that writes o.min_out itself
    c->cp_marked = false;    // set by a kernel that fills the Clopper-Pearson memo itself
    if (c->D.stat == CSE_STAT_ONE_ARM_Z || c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z)
        return cse_launch_sim_ztest(c, P.T, P.NA, P.k_stride, P.K_tiles, lambda, o, s);
    if (c->D.stat == CSE_STAT_BAYES4)
        return cse_launch_sim_bayes4(c, P.T, P.NA, P.k_stride, P.K_tiles, lambda, o, s);
    if (c->D.stat == CSE_STAT_BERRY4)
        return cse_launch_sim_basket(c, P.T, P.NA, P.k_stride, P.K_tiles, lambda, o, s);
    return CSE_UNSUPPORTED_DESIGN;
}

}  // namespace

void cse_prof_begin(cse_ctx* c, int kid, cudaStream_t s)
{
    if (!c || !c->prof_on) return;
    c->prof_skip = c->prof_only >= 0 && kid != c->prof_only;
    if (c->prof_skip) return;
    ProfRec r;
    r.kid = kid;
    r.a = prof_event(c);
    r.b = prof_event(c);
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    c->prof_pending.push_back(r);
}

void cse_prof_end(cse_ctx* c, cudaStream_t s)
{
    if (!c || !c->prof_on || c->prof_skip || c->prof_pending.empty()) return;
    cudaEventRecord(c->prof_pending.back().b, s);
}

extern "C" {

int cse_reseed(cse_ctx* c, uint64_t seed, cse_stream_t stream)
{
    (void)stream;
    if (!c) return CSE_INVALID_ARG;
    c->seed = seed;
    c->u_stale = true;   // regenerated by the next simulating call (launch_tables)
    return CSE_OK;
}

int cse_autotune(cse_ctx* c, const cse_tiles* t, double lambda, double alpha, int32_t* threads_out,
                 int32_t* tiles_out, cse_stream_t stream)
{
    if (!(alpha > 0.0 && alpha < 1.0)) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (c && cse_posterior_design(c->D.stat)) {   // one configuration for the four-arm kernels
        // the packed form of the four-arm selection design runs 512 threads a block
        const bool packed = c->D.stat == CSE_STAT_BAYES4 && c->bt_packed && !c->bt_direct;
        if (threads_out) *threads_out = packed ? 512 : 256;
        if (tiles_out) *tiles_out = 1;
        return CSE_OK;
    }
    Prepared P;
    CSE_TRY(prepare_args(c, t, &P));
    CSE_TRY(tables_and_alpha_prime(c, P, alpha, c->aprime, s));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    const bool prof = c->prof_on;
    c->prof_on = false;
    // the cell-histogram kernel: its (threads, tiles) configurations; the plain
    // path's per-sim kernel: its block sizes
    const bool cells = !c->plain && c->cells_ok;
    int* knob = cells ? &c->cells_cfg : &c->sim_topt;
    const int n_opts = cells ? cse_cells_configs() : 3;
    const int saved = *knob;
    float best = INFINITY;
    int choice = saved;
    int st = CSE_OK;
    SimOut o = {c->sig, c->R, nullptr, nullptr, c->lam_tile, c->ksel};
    for (int opt = 0; opt < n_opts && st == CSE_OK; ++opt) {
        *knob = opt;
        st = sim_pass(c, P, lambda, o, s);                 // warm-up run of this variant
        float total = 0.0f;
        for (int rep = 0; rep < 2 && st == CSE_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = sim_pass(c, P, lambda, o, s);
            cudaEventRecord(e1, s);
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = CSE_CUDA_ERROR;
            total += ms;
        }
        if (st == CSE_OK && total < best) {
            best = total;
            choice = opt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    c->prof_on = prof;
    *knob = (st == CSE_OK) ? choice : saved;
    if (cells) {
        cse_cells_config(c->cells_cfg, threads_out, tiles_out);
    } else {
        if (threads_out) *threads_out = 128 << c->sim_topt;
        if (tiles_out) *tiles_out = 1;
    }
    return st;
}

int cse_set_option(cse_ctx* c, int option, int64_t value)
{
    if (!c) return CSE_INVALID_ARG;
    switch (option) {
    case CSE_OPT_PLAIN:
        c->plain = value != 0;
        if (cse_posterior_design(c->D.stat) && c->bt_tables) c->bt_direct = c->plain;
        return CSE_OK;
    case CSE_OPT_SIM_THREADS: {   // 64, 128, 256 or 512: the z-test simulation kernels' block size
        if (cse_posterior_design(c->D.stat)) return CSE_INVALID_ARG;
        const int cfg = cse_cells_config_index((int)value, 1);
        if (cfg < 0) return CSE_INVALID_ARG;
        c->cells_cfg = cfg;   // one tile per block
        if (value == 128) c->sim_topt = 0;
        else if (value == 256) c->sim_topt = 1;
        else if (value == 512) c->sim_topt = 2;
        return CSE_OK;
    }
    case CSE_OPT_SIM_TILES: {   // tiles a block of the cell kernel works on at once
        if (cse_posterior_design(c->D.stat)) return CSE_INVALID_ARG;
        int nt = 0;
        cse_cells_config(c->cells_cfg, &nt, nullptr);
        const int cfg = cse_cells_config_index(nt, (int)value);
        if (cfg < 0) return CSE_INVALID_ARG;
        c->cells_cfg = cfg;
        return CSE_OK;
    }
    case CSE_OPT_CELLS_BOX: {   // histogram capacity of the cell kernel (0: the allocated one)
        if (cse_posterior_design(c->D.stat)) return CSE_INVALID_ARG;
        const int64_t row = (c->D.stat == CSE_STAT_TWO_ARM_POOLED_Z) ? (int64_t)c->D.n_max + 1 : 1;
        const int64_t cap = c->n_cells < CSE_CELLS_BOX / 2 ? c->n_cells : CSE_CELLS_BOX / 2;
        if (value != 0 && (value < row || value > cap)) return CSE_INVALID_ARG;
        c->cells_box = (int32_t)value;
        return CSE_OK;
    }
    case CSE_OPT_PDL:
        if (value != 0 && value != 1) return CSE_INVALID_ARG;
        c->pdl = value != 0;
        return CSE_OK;
    case CSE_OPT_BAYES_DIRECT:
        if (!cse_posterior_design(c->D.stat)) return CSE_INVALID_ARG;
        if (!value && !c->bt_tables) return CSE_UNSUPPORTED_DESIGN;
        c->bt_direct = value != 0;
        return CSE_OK;
    default:
        return CSE_INVALID_ARG;
    }
}

int cse_profile_enable(cse_ctx* c, int enable)
{
    if (!c) return CSE_INVALID_ARG;
    c->prof_on = enable != 0;
    return CSE_OK;
}

int cse_profile_only(cse_ctx* c, const char* name)
{
    if (!c) return CSE_INVALID_ARG;
    if (!name || !name[0]) {
        c->prof_only = -1;
        return CSE_OK;
    }
    for (int k = 0; k < KID_COUNT; ++k)
        if (strcmp(name, kKernelNames[k]) == 0) {
            c->prof_only = k;
            return CSE_OK;
        }
    return CSE_INVALID_ARG;
}

int cse_profile_read(cse_ctx* c, const char** names, int64_t* launches, double* total_ms, int max)
{
    if (!c || max < 0) return CSE_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    for (auto& r : c->prof_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.kid] += ms;
            c->prof_n[r.kid] += 1;
        }
        cudaGetLastError();
        c->prof_free.push_back(r.a);
        c->prof_free.push_back(r.b);
    }
    c->prof_pending.clear();
    int n = 0;
    for (int k = 0; k < KID_COUNT; ++k) {
        if (c->prof_n[k] == 0) continue;
        if (n < max) {
            if (names) names[n] = kKernelNames[k];
            if (launches) launches[n] = c->prof_n[k];
            if (total_ms) total_ms[n] = c->prof_ms[k];
        }
        ++n;
        c->prof_n[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    return n;
}

const char* cse_status_str(int status)
{
    switch (status) {
    case CSE_OK: return "ok";
    case CSE_INVALID_ARG: return "invalid argument";
    case CSE_UNSUPPORTED_DESIGN: return "unsupported design";
    case CSE_OOM: return "device allocation failed";
    case CSE_CUDA_ERROR: return "CUDA error";
    case CSE_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case CSE_DEVICE_CHECK: return "device-side argument check failed";
    case CSE_CAPACITY: return "request exceeds the fixed scratch capacity";
    default: return "unknown status";
    }
}

int cse_create(cse_ctx** out, const cse_design* design, uint64_t seed, int32_t K_max, cse_stream_t stream)
{
    if (!out || !design) return CSE_INVALID_ARG;
    *out = nullptr;
    if (K_max < 1 || K_max > CSE_MAX_KMAX) return CSE_INVALID_ARG;
    const cse_design& ds = *design;
    if (ds.n_looks < 1 || ds.n_looks > CSE_MAX_LOOKS) return CSE_UNSUPPORTED_DESIGN;
    int prev = 0;
    for (int l = 0; l < ds.n_looks; ++l) {
        if (ds.look_n[l] <= prev) return CSE_UNSUPPORTED_DESIGN;
        prev = ds.look_n[l];
    }
    const int n_max = ds.look_n[ds.n_looks - 1];
    if (n_max > CSE_MAX_NMAX) return CSE_UNSUPPORTED_DESIGN;
    switch (ds.stat) {
    case CSE_STAT_ONE_ARM_Z:
        if (ds.d != 1 || ds.n_looks != 1 || !(ds.p0 > 0.0 && ds.p0 < 1.0)) return CSE_UNSUPPORTED_DESIGN;
        break;
    case CSE_STAT_TWO_ARM_POOLED_Z:
        if (ds.d != 2 || ds.n_looks != 1) return CSE_UNSUPPORTED_DESIGN;
        break;
    case CSE_STAT_BAYES4:
        if (ds.d != 4 || ds.n_looks != 3 || !(ds.drop >= 0.0 && ds.drop <= 1.0)) return CSE_UNSUPPORTED_DESIGN;
        if (ds.look_n[2] > 255) return CSE_UNSUPPORTED_DESIGN;
        break;
    case CSE_STAT_BERRY4:
        if (ds.d != 4 || ds.n_looks != 1 || n_max > 63) return CSE_UNSUPPORTED_DESIGN;
        for (int a = 0; a < 4; ++a)
            if (!isfinite(ds.arm_null[a])) return CSE_UNSUPPORTED_DESIGN;
        break;
    default:
        return CSE_UNSUPPORTED_DESIGN;
    }
    cse_ctx* c = new (std::nothrow) cse_ctx();
    if (!c) return CSE_OOM;
    c->D.stat = ds.stat;
    c->D.d = ds.d;
    c->D.n_looks = ds.n_looks;
    for (int l = 0; l < CSE_MAX_LOOKS; ++l) c->D.look_n[l] = (l < ds.n_looks) ? ds.look_n[l] : n_max;
    c->D.n_max = n_max;
    c->D.p0 = ds.p0;
    c->D.drop = ds.drop;
    for (int a = 0; a < CSE_MAX_ARMS; ++a) c->D.tnull[a] = (ds.stat == CSE_STAT_BERRY4) ? ds.arm_null[a] : 0.0;
    c->seed = seed;
    c->K_max = K_max;
    c->sim_topt = 0;   // 128 threads until cse_autotune chooses
    c->pdl = false;   // measured: faster only where launch latency dominates (CSE_OPT_PDL)
    cudaGetDevice(&c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int st = CSE_OK;
    do {
        const size_t ub = sizeof(uint32_t) * (size_t)ds.d * (size_t)K_max * (size_t)n_max;
        if (cudaMalloc(&c->U, ub) != cudaSuccess) { st = CSE_OOM; break; }
        if (cudaMalloc(&c->tb, sizeof(uint32_t) * (size_t)K_max) != cudaSuccess) { st = CSE_OOM; break; }
        if (ds.stat == CSE_STAT_ONE_ARM_Z) {
            c->n_cells = n_max + 1;
            c->n1p = 1;
        } else if (ds.stat == CSE_STAT_TWO_ARM_POOLED_Z) {
            c->n1p = n_max + 1;
            c->n_cells = (n_max + 1) * (n_max + 1);
        }
        if (c->n_cells > 0) {
            if (cudaMalloc(&c->S_tab, 4 * (size_t)c->n_cells) != cudaSuccess ||
                cudaMalloc(&c->rank_tab, 2 * (size_t)c->n_cells) != cudaSuccess ||
                cudaMalloc(&c->val_of_rank, 4 * (size_t)c->n_cells) != cudaSuccess ||
                cudaMalloc(&c->cell_of_pos, 8 * (size_t)c->n_cells) != cudaSuccess) { st = CSE_OOM; break; }
        }
        if (cudaMalloc(&c->counter, 64) != cudaSuccess || cudaMalloc(&c->err, 64) != cudaSuccess ||
            cudaMalloc(&c->cp_nkeys, 64) != cudaSuccess || cudaMalloc(&c->min_key, 64) != cudaSuccess ||
            cudaMalloc(&c->lam_dev, 64) != cudaSuccess) { st = CSE_OOM; break; }
        if (cudaMallocHost(&c->lam_host, 64) != cudaSuccess) { st = CSE_OOM; break; }
        if (cudaMallocHost(&c->pt_count_host, 64) != cudaSuccess) { st = CSE_OOM; break; }
        if (cudaMalloc(&c->pt_count, 64) != cudaSuccess) { st = CSE_OOM; break; }
        if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            st = CSE_CUDA_ERROR;
            break;
        }
        if (cse_bound_set_attrs() != CSE_OK) {
            st = CSE_CUDA_ERROR;
            break;
        }
        // initial states that the kernels restore after each use: work-queue head and
        // ticket 0, key count 0, running-minimum key all ones and its ticket 0
        if (cudaMemsetAsync(c->err, 0, 64, s) != cudaSuccess || cudaMemsetAsync(c->min_key, 0, 64, s) != cudaSuccess ||
            cudaMemsetAsync(c->min_key, 0xFF, sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemsetAsync(c->counter, 0, 64, s) != cudaSuccess || cudaMemsetAsync(c->cp_nkeys, 0, 64, s) != cudaSuccess) {
            st = CSE_CUDA_ERROR;
            break;
        }
        c->min_ticket = reinterpret_cast<unsigned int*>(c->min_key + 1);
        st = cse_launch_uniforms(c, s);
        if (st != CSE_OK) break;
        st = cse_launch_tables(c, s);
        if (st != CSE_OK) break;
        if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            st = CSE_CUDA_ERROR;
            break;
        }
        if (ds.stat == CSE_STAT_BAYES4) {
            st = cse_bayes4_setup(c, s);
        } else if (ds.stat == CSE_STAT_BERRY4) {
            st = cse_basket_setup(c, s);
        } else {
            st = cse_sim_ztest_setup(c);
        }
        if (st != CSE_OK) break;
        if (cudaStreamSynchronize(s) != cudaSuccess) st = CSE_CUDA_ERROR;
    } while (0);
    if (st != CSE_OK) {
        cudaGetLastError();
        cse_destroy(c);
        return st;
    }
    *out = c;
    return CSE_OK;
}

int cse_destroy(cse_ctx* c)
{
    if (!c) return CSE_OK;
    cudaDeviceSynchronize();
    cudaFree(c->U);
    cudaFree(c->tb);
    cudaFree(c->tbuf);
    cudaFree(c->S_tab);
    cudaFree(c->rank_tab);
    cudaFree(c->val_of_rank);
    cudaFree(c->cell_of_pos);
    cudaFree(c->xs);
    cudaFree(c->tie_rm);
    cudaFree(c->thr);
    cudaFree(c->sig);
    cudaFree(c->cnt);
    cudaFree(c->bb);
    cudaFree(c->ksel);
    cudaFree(c->aprime);
    cudaFree(c->lam_tile);
    cudaFree(c->R);
    cudaFree(c->cp_key);
    cudaFree(c->cp_val);
    cudaFree(c->cp_slot);
    cudaFree(c->cp_list);
    cudaFree(c->cp_nkeys);
    cudaFree(c->min_key);
    cudaFree(c->geom);
    cudaFree(c->bt_d1);
    cudaFree(c->bt_d2);
    cudaFree(c->bt_d2s);
    cudaFree(c->bt_f4);
    cudaFree(c->bk_q);
    cudaFree(c->keys);
    cudaFree(c->counter);
    cudaFree(c->err);
    cudaFree(c->lam_dev);
    if (c->lam_host) cudaFreeHost(c->lam_host);
    if (c->pt_count_host) cudaFreeHost(c->pt_count_host);
    cudaFree(c->pt_count);
    cudaFree(c->pt_keys);
    cudaFree(c->pt_vals);
    cudaFree(c->pt_axis);
    cudaFree(c->pt_idx);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto& r : c->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof_free) cudaEventDestroy(e);
    cudaGetLastError();
    delete c;
    return CSE_OK;
}

int cse_simulate_tiles(cse_ctx* c, const cse_tiles* t, double lambda, int64_t* R_out, int64_t* Xrej_out,
                       double* score_out, cse_stream_t stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    SimOut o = {c->sig, R_out, Xrej_out, score_out, nullptr, nullptr};
    return sim_pass(c, P, lambda, o, s);
}

int cse_type1_error(cse_ctx* c, int64_t n_points, const double* theta, const uint32_t* null_mask, const int32_t* K,
                    int32_t K_max, double lambda, double* fhat_out, int64_t* R_out, int64_t* Xrej_out,
                    double* score_out, cse_stream_t stream)
{
    if (!c || n_points < 1 || !theta || !null_mask || !K || !fhat_out) return CSE_INVALID_ARG;
    if (K_max < 1 || K_max > c->K_max || n_points > ((int64_t)1 << 28)) return CSE_INVALID_ARG;
    const int d = c->D.d;
    cudaStream_t s = (cudaStream_t)stream;
    if ((size_t)n_points > c->pt_cap) {
        cudaFree(c->pt_keys);
        cudaFree(c->pt_vals);
        cudaFree(c->pt_axis);
        cudaFree(c->pt_idx);
        c->pt_keys = nullptr;
        c->pt_vals = nullptr;
        c->pt_axis = nullptr;
        c->pt_idx = nullptr;
        c->pt_cap = 0;
        uint32_t P = 1024;
        while ((int64_t)P < 2 * n_points) P <<= 1;
        const size_t n = (size_t)n_points;
        if (cudaMalloc(&c->pt_keys, sizeof(unsigned long long) * CSE_MAX_ARMS * P) != cudaSuccess ||
            cudaMalloc(&c->pt_vals, sizeof(int32_t) * CSE_MAX_ARMS * P) != cudaSuccess ||
            cudaMalloc(&c->pt_axis, sizeof(double) * CSE_MAX_ARMS * n) != cudaSuccess ||
            cudaMalloc(&c->pt_idx, sizeof(int32_t) * CSE_MAX_ARMS * n) != cudaSuccess) {
            cudaGetLastError();
            return CSE_OOM;
        }
        c->pt_P = P;
        c->pt_cap = n;
    }
    // distinct coordinates per arm, then their number back on the host (it sizes
    // the count tables)
    CSE_TRY(cse_launch_point_axes(c, theta, n_points, d, s));
    CUDA_TRY(cudaMemcpyAsync(c->pt_count_host, c->pt_count, sizeof(int32_t) * CSE_MAX_ARMS, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    cse_tiles t;
    memset(&t, 0, sizeof(t));
    t.n_tiles = n_points;
    for (int a = 0; a < d; ++a) {
        t.n_axis[a] = c->pt_count_host[a];
        t.axis[a] = c->pt_axis + (size_t)a * c->pt_cap;
    }
    t.center_idx = c->pt_idx;
    t.halfwidth = nullptr;   // the simulation reads no half-widths
    t.null_mask = null_mask;
    t.K = K;
    t.K_max = K_max;
    Prepared P;
    CSE_TRY(prepare(c, &t, s, &P, false));
    int64_t* R = R_out ? R_out : c->R;
    SimOut o = {c->sig, R, Xrej_out, score_out, nullptr, nullptr};
    CSE_TRY(sim_pass(c, P, lambda, o, s));
    return cse_launch_fhat(c, R, K, n_points, fhat_out, s);
}

int cse_validate(cse_ctx* c, const cse_tiles* t, double lambda, double delta, int64_t* R_out,
                 int64_t* Xrej_out, double* score_out, double* u0_out, double* bound_out, double* qstar_out,
                 cse_stream_t stream)
{
    if (!(delta > 0.0 && delta < 1.0)) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    int64_t* R = R_out ? R_out : c->R;
    SimOut o = {c->sig, R, Xrej_out, score_out, nullptr, nullptr};
    CSE_TRY(sim_pass(c, P, lambda, o, s));
    return cse_launch_bounds(c, P.T, R, delta, false, u0_out, bound_out, qstar_out, s);
}

int cse_validate_lower(cse_ctx* c, const cse_tiles* t, double lambda, double delta, int64_t* R_out,
                       int64_t* Xrej_out, double* score_out, double* l0_out, double* lower_out, double* qstar_out,
                       cse_stream_t stream)
{
    if (!(delta > 0.0 && delta < 1.0)) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    int64_t* R = R_out ? R_out : c->R;
    SimOut o = {c->sig, R, Xrej_out, score_out, nullptr, nullptr};
    CSE_TRY(sim_pass(c, P, lambda, o, s));
    return cse_launch_bounds(c, P.T, R, delta, true, l0_out, lower_out, qstar_out, s);
}

int cse_validate_band(cse_ctx* c, const cse_tiles* t, double lambda, double delta, int64_t* R_out,
                      int64_t* Xrej_out, double* score_out, double* l0_out, double* lower_out, double* u0_out,
                      double* upper_out, cse_stream_t stream)
{
    if (!(delta > 0.0 && delta < 1.0)) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    int64_t* R = R_out ? R_out : c->R;
    SimOut o = {c->sig, R, Xrej_out, score_out, nullptr, nullptr};
    CSE_TRY(sim_pass(c, P, lambda, o, s));
    // each side at delta / 2: both hold together with probability >= 1 - delta
    CSE_TRY(cse_launch_bounds(c, P.T, R, 0.5 * delta, true, l0_out, lower_out, nullptr, s));
    return cse_launch_bounds(c, P.T, R, 0.5 * delta, false, u0_out, upper_out, nullptr, s);
}

int cse_validate_rand(cse_ctx* c, const cse_tiles* t, double lambda, uint32_t c_thr, double delta, int64_t* R_out,
                      int64_t* Xrej_out, double* score_out, double* u0_out, double* bound_out, double* qstar_out,
                      cse_stream_t stream)
{
    if (!(delta > 0.0 && delta < 1.0)) return CSE_INVALID_ARG;
    if (c && cse_posterior_design(c->D.stat)) return CSE_UNSUPPORTED_DESIGN;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    int64_t* R = R_out ? R_out : c->R;
    SimOut o = {c->sig, R, Xrej_out, score_out, nullptr, nullptr};
    CSE_TRY(cse_launch_sim_rand(c, P.T, P.NA, P.k_stride, P.K_tiles, lambda, c_thr, o, nullptr, s));
    return cse_launch_bounds(c, P.T, R, delta, false, u0_out, bound_out, qstar_out, s);
}

int cse_calibrate_rand(cse_ctx* c, const cse_tiles* t, double alpha, double* alpha_prime_out,
                       double* lambda_tile_out, uint32_t* c_tile_out, double* lambda_out, uint32_t* c_out,
                       cse_stream_t stream)
{
    if (!(alpha > 0.0 && alpha < 1.0)) return CSE_INVALID_ARG;
    if (!lambda_tile_out || !c_tile_out) return CSE_INVALID_ARG;
    if (c && cse_posterior_design(c->D.stat)) return CSE_UNSUPPORTED_DESIGN;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare_args(c, t, &P));
    CSE_TRY(tables_and_alpha_prime(c, P, alpha, alpha_prime_out, s));
    SimOut o = {c->sig, nullptr, nullptr, nullptr, lambda_tile_out, c->ksel};
    CSE_TRY(cse_launch_sim_rand(c, P.T, P.NA, P.k_stride, P.K_tiles, INFINITY, 0u, o, c_tile_out, s));
    // (lambda*, c*) through the device scalars lam_dev and lam_dev + 1 (its low 4 bytes)
    uint32_t* c_dev = reinterpret_cast<uint32_t*>(c->lam_dev + 1);
    CSE_TRY(cse_launch_min_pair(c, lambda_tile_out, c_tile_out, t->n_tiles, c->lam_dev, c_dev, s));
    CUDA_TRY(cudaMemcpyAsync(c->lam_host, c->lam_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (lambda_out) *lambda_out = c->lam_host[0];
    if (c_out) *c_out = *reinterpret_cast<const uint32_t*>(c->lam_host + 1);
    return cse_sync(c, stream);
}

int cse_calibrate(cse_ctx* c, const cse_tiles* t, double alpha, double* alpha_prime_out,
                  double* lambda_tile_out, double* lambda_out, cse_stream_t stream)
{
    if (!(alpha > 0.0 && alpha < 1.0)) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare_args(c, t, &P));
    double* lam_tile = lambda_tile_out ? lambda_tile_out : c->lam_tile;
    CSE_TRY(tables_and_alpha_prime(c, P, alpha, alpha_prime_out, s));
    SimOut o = {c->sig, nullptr, nullptr, nullptr, lam_tile, c->ksel};
    o.min_key = c->min_key;
    o.min_out = c->lam_dev;
    CSE_TRY(sim_pass(c, P, INFINITY, o, s));
    if (!c->min_folded) CSE_TRY(cse_launch_min(c, lam_tile, t->n_tiles, c->lam_dev, s));
    CUDA_TRY(cudaMemcpyAsync(c->lam_host, c->lam_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (lambda_out) *lambda_out = *c->lam_host;
    return cse_sync(c, stream);
}

int cse_step(cse_ctx* c, const cse_tiles* t, double lambda, double delta, double alpha, int64_t* R_out,
             int64_t* Xrej_out, double* score_out, double* u0_out, double* bound_out, double* qstar_out,
             double* alpha_prime_out, double* lambda_tile_out, double* lambda_dev, cse_stream_t stream)
{
    if (!(delta > 0.0 && delta < 1.0) || !(alpha > 0.0 && alpha < 1.0)) return CSE_INVALID_ARG;
    if (!lambda_tile_out || !lambda_dev) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare_args(c, t, &P));
    int64_t* R = R_out ? R_out : c->R;
    // alpha' leaves each tile's per-arm softplus terms for the bound pass
    double* geom = nullptr;
    if (!c->plain) {
        CSE_TRY(grow((void**)&c->geom, &c->geom_cap, sizeof(double) * 3 * (size_t)P.T.d * (size_t)t->n_tiles));
        geom = c->geom;
    }
    CSE_TRY(tables_and_alpha_prime(c, P, alpha, alpha_prime_out, s, geom));
    SimOut o = {c->sig, R, Xrej_out, score_out, lambda_tile_out, c->ksel};
    o.min_key = c->min_key;   // the simulation kernel folds the minimum over tiles where it can
    o.min_out = lambda_dev;
    if (!c->plain && c->cp_cap >= 2 * (uint64_t)t->n_tiles) {   // and the memo's key insertion
        o.cp_key = c->cp_key;
        o.cp_cap = (uint32_t)c->cp_cap;
        o.cp_slot = c->cp_slot;
        o.cp_list = c->cp_list;
        o.cp_nkeys = c->cp_nkeys;
    }
    CSE_TRY(sim_pass(c, P, lambda, o, s));
    CSE_TRY(cse_launch_bounds(c, P.T, R, delta, false, u0_out, bound_out, qstar_out, s, geom, c->cp_marked));
    if (c->min_folded) return CSE_OK;
    return cse_launch_min(c, lambda_tile_out, t->n_tiles, lambda_dev, s);
}

int cse_statistics(cse_ctx* c, const cse_tiles* t, const int64_t* offsets, float* S_out, cse_stream_t stream)
{
    if (!offsets || !S_out) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Prepared P;
    CSE_TRY(prepare(c, t, s, &P));
    if (c->plain && !cse_posterior_design(c->D.stat))   // the export reads the axis count table
        CSE_TRY(cse_launch_axis_counts(c, P.T, P.NA, P.K_tiles, P.k_stride, s));
    if (c->D.stat == CSE_STAT_BAYES4)
        return cse_launch_emit_bayes4(c, P.T, P.NA, P.k_stride, P.K_tiles, offsets, S_out, s);
    if (c->D.stat == CSE_STAT_BERRY4)
        return cse_launch_emit_basket(c, P.T, P.NA, P.k_stride, P.K_tiles, offsets, S_out, s);
    return cse_launch_emit_ztest(c, P.T, P.NA, P.k_stride, P.K_tiles, offsets, S_out, s);
}

int cse_score_backward(int64_t n_tiles, int32_t d, const double* grad_out, const double* score, const int32_t* K,
                       double* grad_theta, cse_stream_t stream)
{
    if (n_tiles < 0 || d < 1 || d > CSE_MAX_ARMS) return CSE_INVALID_ARG;
    if (n_tiles > 0 && (!grad_out || !score || !K || !grad_theta)) return CSE_INVALID_ARG;
    return cse_launch_backward(n_tiles, d, grad_out, score, K, grad_theta, (cudaStream_t)stream);
}

int cse_sync(cse_ctx* c, cse_stream_t stream)
{
    if (!c) return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t flags = 0;
    if (cudaMemcpyAsync(&flags, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    if (flags) {
        cudaMemsetAsync(c->err, 0, sizeof(int32_t), s);
        cudaStreamSynchronize(s);
        return (flags & CSE_ERR_TIMEOUT) ? CSE_DEVICE_TIMEOUT : CSE_DEVICE_CHECK;
    }
    return CSE_OK;
}

int64_t cse_launch_count(const cse_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"

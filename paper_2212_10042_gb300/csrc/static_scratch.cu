// static_scratch.cu -- an allocation-free variant of the z-test simulation.
//
// Some callers cannot allocate device memory: a plugin inside a host program
// that owns and accounts for all GPU memory, or a loop that must not stall,
// since cudaMalloc/cudaFree can synchronise the device.  For them,
// cse_simulate_tiles_static runs the same kernels as cse_create +
// cse_simulate_tiles, but every scratch buffer (CRN uniforms, thresholds, the
// axis count table, statistic tables, work counter, error flag) is carved out
// of one fixed array in device global memory, declared below.  Every GPU that
// loads this library holds that array until the process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "cse_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB, see include/cse.h

// The scratch.  Host code must not pass this name to a kernel (on the host it
// is only a stand-in object); it uses the device address returned by
// cudaGetSymbolAddress instead.  Shared by every call: it keeps the previous
// call's contents, and calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_cse_scratch[kStaticScratchBytes];

std::mutex g_mutex;
std::vector<void*> g_scratch_addr;   // per device ordinal, sized from cudaGetDeviceCount

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr.empty()) {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
            cudaGetLastError();
            return CSE_CUDA_ERROR;
        }
        g_scratch_addr.assign((size_t)n, nullptr);
    }
    if (dev < 0 || dev >= (int)g_scratch_addr.size()) return CSE_CUDA_ERROR;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cse_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CSE_CUDA_ERROR;
        }
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_addr[dev];
    return CSE_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int cse_simulate_tiles_static(const cse_design* design, uint64_t seed, const cse_tiles* t,
                                         double lambda, int64_t* R_out, int64_t* Xrej_out, double* score_out,
                                         cse_stream_t stream)
{
    if (!design || !t) return CSE_INVALID_ARG;
    const cse_design& ds = *design;
    if (ds.stat != CSE_STAT_ONE_ARM_Z && ds.stat != CSE_STAT_TWO_ARM_POOLED_Z) return CSE_UNSUPPORTED_DESIGN;
    if (ds.n_looks != 1 || ds.look_n[0] < 1 || ds.look_n[0] > CSE_MAX_NMAX) return CSE_UNSUPPORTED_DESIGN;
    if (ds.stat == CSE_STAT_ONE_ARM_Z && (ds.d != 1 || !(ds.p0 > 0.0 && ds.p0 < 1.0))) return CSE_UNSUPPORTED_DESIGN;
    if (ds.stat == CSE_STAT_TWO_ARM_POOLED_Z && ds.d != 2) return CSE_UNSUPPORTED_DESIGN;
    if (t->n_tiles < 1 || !t->center_idx || !t->halfwidth || !t->null_mask || !t->K) return CSE_INVALID_ARG;
    if (t->K_max < 1 || t->K_max > CSE_MAX_KMAX) return CSE_INVALID_ARG;

    // a context on the host stack whose device buffers all live in the scratch
    cse_ctx c{};
    const int n_max = ds.look_n[0];
    c.D.stat = ds.stat;
    c.D.d = ds.d;
    c.D.n_looks = 1;
    for (int l = 0; l < CSE_MAX_LOOKS; ++l) c.D.look_n[l] = n_max;
    c.D.n_max = n_max;
    c.D.p0 = ds.p0;
    c.D.drop = ds.drop;
    c.seed = seed;
    c.K_max = t->K_max;
    c.sim_topt = 1;
    c.n1p = (ds.stat == CSE_STAT_TWO_ARM_POOLED_Z) ? n_max + 1 : 1;
    c.n_cells = (ds.stat == CSE_STAT_TWO_ARM_POOLED_Z) ? (n_max + 1) * (n_max + 1) : n_max + 1;

    TileArgs T;
    memset(&T, 0, sizeof(T));
    T.n_tiles = t->n_tiles;
    T.d = ds.d;
    int32_t na = 0;
    for (int a = 0; a < ds.d; ++a) {
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
    const int32_t k_stride = (t->K_max + 15) / 16 * 16;

    // layout of the scratch
    const size_t off_flags = 0;                                   // counter, error flag
    const size_t off_U = 256;
    const size_t sz_U = sizeof(uint32_t) * (size_t)ds.d * (size_t)t->K_max * (size_t)n_max;
    const size_t off_thr = off_U + align256(sz_U);
    const size_t off_sig = off_thr + align256(sizeof(uint32_t) * (size_t)na);
    const size_t off_cnt = off_sig + align256(sizeof(double) * (size_t)na);
    const size_t off_S = off_cnt + align256((size_t)na * (size_t)k_stride);
    const size_t off_rank = off_S + align256(4 * (size_t)c.n_cells);
    const size_t off_vor = off_rank + align256(2 * (size_t)c.n_cells);
    const size_t off_bb = off_vor + align256(4 * (size_t)c.n_cells);
    const size_t total = off_bb + align256(sizeof(uint32_t) * 2 * (size_t)na);
    if (total > kStaticScratchBytes) return CSE_CAPACITY;

    cudaStream_t s = (cudaStream_t)stream;
    // the call ends with a copy of the error flag to the host and a stream
    // synchronisation, which a stream capture cannot hold: refuse it before any
    // other CUDA call rather than invalidate the caller's capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    if (cap != cudaStreamCaptureStatusNone) return CSE_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    unsigned char* base = nullptr;
    int st = scratch_address(dev, &base);
    if (st != CSE_OK) return st;
    c.device = dev;
    c.counter = (int32_t*)(base + off_flags);
    c.err = (int32_t*)(base + off_flags + 64);
    c.U = (uint32_t*)(base + off_U);
    c.thr = (uint32_t*)(base + off_thr);
    c.sig = (double*)(base + off_sig);
    c.cnt = base + off_cnt;
    c.S_tab = (float*)(base + off_S);
    c.rank_tab = (uint16_t*)(base + off_rank);
    c.val_of_rank = (float*)(base + off_vor);
    c.bb = (uint32_t*)(base + off_bb);
    if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    st = cse_sim_ztest_setup(&c);
    if (st != CSE_OK) return st;

    // the previous call's flags are still in the scratch: clear them first
    if (cudaMemsetAsync(base + off_flags, 0, 256, s) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    if ((st = cse_launch_uniforms(&c, s)) != CSE_OK) return st;
    if ((st = cse_launch_tables(&c, s)) != CSE_OK) return st;
    if ((st = cse_launch_thresholds(&c, T, na, s)) != CSE_OK) return st;
    if ((st = cse_launch_axis_counts(&c, T, na, t->K_max, k_stride, s)) != CSE_OK) return st;
    SimOut o = {c.sig, R_out, Xrej_out, score_out, nullptr, nullptr};
    if ((st = cse_launch_sim_ztest(&c, T, na, k_stride, t->K_max, lambda, o, s)) != CSE_OK) return st;
    int32_t flags = 0;
    if (cudaMemcpyAsync(&flags, c.err, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    return flags ? CSE_DEVICE_CHECK : CSE_OK;
}

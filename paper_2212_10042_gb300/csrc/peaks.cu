// peaks.cu -- measured issue rates of the pipes the simulation kernels use.
//
// Measurement support (the paper has no counterpart): the throughput of a
// kernel on this path is reported as a fraction of what the unit that bounds
// it can do on this GPU, and these probes measure that with CUDA events
// instead of taking it from nominal lane counts.  Each probe keeps every SM
// busy with a long stream of independent instructions of one kind and counts
// them:
//   - ALU pipe: 3-input logic (lop3.b32) on eight interleaved chains;
//   - FP32 FMA pipe: fma.rn.f32 on eight chains;
//   - FP64 pipe: fma.rn.f64 on eight chains;
//   - shared-memory atomics: atom.shared.add.u32 with every lane of a warp on
//     its own bank (the conflict-free rate; the z-test kernels' histogram
//     increments are this instruction).
// Operations are counted per lane: one warp instruction = 32 lane-ops.
#include <cuda_runtime.h>

#include "cse_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kUnroll = 16;   // rounds of eight chains per loop iteration

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t lop3_maj(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// 8 chains x kUnroll rounds x iters lop3 per thread
__global__ void __launch_bounds__(kProbeThreads) k_probe_alu(int32_t iters, uint32_t seed, uint32_t* __restrict__ sink)
{
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (uint32_t)i + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t b = x[(i + 1) & 7], c = x[(i + 3) & 7];
                x[i] = (r & 1) ? lop3_maj(x[i], b, c) : lop3_xor3(x[i], b, c);
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == 0x7FFFFFFFu) sink[0] = acc;   // never in practice; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int32_t iters, float a, float b, float* __restrict__ sink)
{
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = __fmaf_rn(x[i], a, b);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += x[i];
    if (acc == 1234.5f) sink[0] = acc;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(int32_t iters, double a, double b, double* __restrict__ sink)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = __fma_rn(x[i], a, b);
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += x[i];
    if (acc == 1234.5) sink[0] = acc;
}

// each lane adds to words of its own bank: word (j, threadIdx.x) of h sits in
// bank threadIdx.x % 32; eight words per thread, so that consecutive atomics of
// a thread are independent; 8 x kUnroll atomics per iteration
__global__ void __launch_bounds__(kProbeThreads) k_probe_atoms(int32_t iters, uint32_t* __restrict__ sink)
{
    __shared__ uint32_t h[8][kProbeThreads];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j][threadIdx.x] = 0u;
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8 * kUnroll; ++r) atomicAdd(&h[r & 7][threadIdx.x], 1u);
    }
    __syncthreads();
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) ok &= h[j][threadIdx.x] == (uint32_t)iters * kUnroll;
    if (!ok) atomicOr(sink, 1u);   // every increment landed
}

}  // namespace

extern "C" int cse_probe_peak(int kind, int32_t blocks_per_sm, int32_t iters, int32_t reps, double* ops_per_s,
                              double* ms_per_launch, cse_stream_t stream)
{
    if (kind < CSE_PROBE_ALU || kind > CSE_PROBE_SMEM_ATOMIC) return CSE_INVALID_ARG;
    if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (1 << 20) || reps < 1 || reps > 1000)
        return CSE_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    void* sink = nullptr;
    if (cudaMallocAsync(&sink, 64, s) != cudaSuccess || cudaMemsetAsync(sink, 0, 64, s) != cudaSuccess) {
        cudaGetLastError();
        return CSE_OOM;
    }
    const dim3 grid((unsigned)(sms * blocks_per_sm)), block(kProbeThreads);
    auto launch = [&]() {
        switch (kind) {
        case CSE_PROBE_ALU: k_probe_alu<<<grid, block, 0, s>>>(iters, 0x1234567u, (uint32_t*)sink); break;
        case CSE_PROBE_FMA: k_probe_fma<<<grid, block, 0, s>>>(iters, 0.999f, 1e-7f, (float*)sink); break;
        case CSE_PROBE_DFMA: k_probe_dfma<<<grid, block, 0, s>>>(iters, 0.999, 1e-7, (double*)sink); break;
        default: k_probe_atoms<<<grid, block, 0, s>>>(iters, (uint32_t*)sink); break;
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = CSE_OK;
    float ms = 0.0f;
    uint32_t bad = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = CSE_CUDA_ERROR;
    if (st == CSE_OK) {
        launch();   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpyAsync(&bad, sink, sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = CSE_CUDA_ERROR;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    cudaStreamSynchronize(s);
    cudaGetLastError();
    if (st != CSE_OK) return st;
    if (kind == CSE_PROBE_SMEM_ATOMIC && bad) return CSE_DEVICE_CHECK;
    const double per_launch = (double)grid.x * kProbeThreads * (double)iters * 8.0 * kUnroll;
    if (ops_per_s) *ops_per_s = per_launch * reps / (ms * 1e-3);
    if (ms_per_launch) *ms_per_launch = ms / reps;
    return CSE_OK;
}

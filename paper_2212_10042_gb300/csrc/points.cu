// points.cu -- simulation at arbitrary points theta_i (Sec. 6.1): the axis-indexed
// form of a tile set built on the device, and the Monte Carlo estimate
// f_hat_i = R_i / K_i.
//
// The success count of (sim k, arm a) depends on the point only through
// theta_ia (common random numbers, Sec. 7.3), so the simulation runs once per
// distinct coordinate of each arm.  The distinct coordinates are gathered by an
// open-addressing hash table per arm, keyed by the coordinate's 64 bits (every
// NaN folded to one key): the first insert of a key takes the next dense index,
// a second kernel gives every (point, arm) the index of its key.  The order of
// the dense indices depends on the order of the atomic inserts; no result does
// (the count tables are per coordinate and accept any order).
#include <cuda_runtime.h>

#include "cse_internal.cuh"

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;   // a NaN pattern no key takes (NaNs fold to kNanKey)
constexpr unsigned long long kNanKey = 0x7FF8000000000000ull;

__device__ __forceinline__ unsigned long long coord_key(double x)
{
    return isnan(x) ? kNanKey : (unsigned long long)__double_as_longlong(x);
}

__device__ __forceinline__ uint32_t key_hash(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;   // MurmurHash3 fmix64
    k ^= k >> 33;
    return (uint32_t)k;
}

// Insert theta[i*d + a] into arm a's table (keys[a*P ...], P a power of two >
// number of points, so a free slot always exists and the probe ends within P
// steps).  A new key takes dense index atomicAdd(count[a]) and writes its
// coordinate to axis[a*stride + index] (stride >= n).
__global__ void k_point_insert(const double* __restrict__ theta, int64_t n, int32_t d, uint32_t P,
                               unsigned long long* __restrict__ keys, int32_t* __restrict__ vals,
                               int32_t* __restrict__ count, double* __restrict__ axis, int64_t stride)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * d) return;
    const int a = (int)(t % d);
    const double x = theta[t];
    const unsigned long long k = coord_key(x);
    unsigned long long* kt = keys + (int64_t)a * P;
    uint32_t s = key_hash(k) & (P - 1);
    for (uint32_t probe = 0; probe < P; ++probe) {
        const unsigned long long prev = atomicCAS(kt + s, kEmptyKey, k);
        if (prev == kEmptyKey) {
            const int id = atomicAdd(count + a, 1);
            vals[(int64_t)a * P + s] = id;
            axis[(int64_t)a * stride + id] = x;
            return;
        }
        if (prev == k) return;
        s = (s + 1) & (P - 1);
    }
}

// center_idx[i*d + a] = dense index of theta[i*d + a]'s key (after every insert).
__global__ void k_point_index(const double* __restrict__ theta, int64_t n, int32_t d, uint32_t P,
                              const unsigned long long* __restrict__ keys, const int32_t* __restrict__ vals,
                              int32_t* __restrict__ idx)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * d) return;
    const int a = (int)(t % d);
    const unsigned long long k = coord_key(theta[t]);
    const unsigned long long* kt = keys + (int64_t)a * P;
    uint32_t s = key_hash(k) & (P - 1);
    int id = -1;   // not found cannot happen after the insert pass; -1 fails the simulation's index check
    for (uint32_t probe = 0; probe < P; ++probe) {
        const unsigned long long cur = kt[s];
        if (cur == k) {
            id = vals[(int64_t)a * P + s];
            break;
        }
        if (cur == kEmptyKey) break;
        s = (s + 1) & (P - 1);
    }
    idx[t] = id;
}

// f_hat_i = R_i / K_i (Sec. 6.1, the Monte Carlo estimate of the Type I Error).
__global__ void k_fhat(const int64_t* __restrict__ R, const int32_t* __restrict__ K, int64_t n,
                       double* __restrict__ fhat)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    fhat[i] = (double)R[i] / (double)K[i];
}

}  // namespace

int cse_launch_point_axes(cse_ctx* c, const double* theta, int64_t n, int32_t d, cudaStream_t s)
{
    const int64_t nd = n * d;
    const unsigned blocks = (unsigned)((nd + 255) / 256);
    if (cudaMemsetAsync(c->pt_keys, 0xFF, sizeof(unsigned long long) * (size_t)d * c->pt_P, s) != cudaSuccess ||
        cudaMemsetAsync(c->pt_count, 0, sizeof(int32_t) * CSE_MAX_ARMS, s) != cudaSuccess) {
        cudaGetLastError();
        return CSE_CUDA_ERROR;
    }
    k_point_insert<<<blocks, 256, 0, s>>>(theta, n, d, c->pt_P, c->pt_keys, c->pt_vals, c->pt_count, c->pt_axis,
                                          (int64_t)c->pt_cap);
    k_point_index<<<blocks, 256, 0, s>>>(theta, n, d, c->pt_P, c->pt_keys, c->pt_vals, c->pt_idx);
    c->launches += 2;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

int cse_launch_fhat(cse_ctx* c, const int64_t* R, const int32_t* K, int64_t n, double* fhat, cudaStream_t s)
{
    k_fhat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, K, n, fhat);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? CSE_OK : CSE_CUDA_ERROR;
}

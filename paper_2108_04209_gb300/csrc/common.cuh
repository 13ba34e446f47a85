// Shared device/host helpers of the SuperDC GB300 library (sm_103a, FP64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "superdc.h"
#include "check.cuh"

#define SDC_EPS 2.220446049250313080847263336181640625e-16   // 2^-52

#define SDC_CHECK(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return (e_ == cudaErrorMemoryAllocation)        \
                                   ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA;       \
    } while (0)

__device__ __forceinline__ void sdc_latch(int32_t *status, int bits)
{
    if (status) atomicOr(status, bits);
}

// largest p in [0, n) with a[p] <= x (a ascending, a[0] <= x)
template <typename T>
__device__ __forceinline__ int64_t sdc_upper_index(const T *__restrict__ a, int64_t n, T x)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Number of SMs of the current device (cached per device by the caller).
int sdc_num_sms();

// Test hook of superdc_debug_alloc_limit: true when an allocation of this
// many bytes must fail as if the device were out of memory.
bool sdc_alloc_denied(size_t bytes);

// The library's stream-ordered memory pool on the current device (created on
// first use): freed scratch stays in the pool across synchronisations (up to
// SDC_POOL_KEEP bytes), so a call after a synchronising one does not map its
// scratch again (the device's default pool returns everything to the driver
// at every synchronisation).  NULL if the pool cannot be created (then the
// default pool serves).
cudaMemPool_t sdc_pool();
constexpr unsigned long long SDC_POOL_KEEP = 16ull << 30;

// Stream-ordered scratch allocation helpers.
template <typename T>
static inline cudaError_t sdc_alloc(T **p, size_t count, cudaStream_t st)
{
    if (count == 0) count = 1;
    if (sdc_alloc_denied(count * sizeof(T))) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = sdc_pool();
    if (pool) return cudaMallocFromPoolAsync((void **)p, count * sizeof(T), pool, st);
    return cudaMallocAsync((void **)p, count * sizeof(T), st);
}

// Synchronous allocation (handles that outlive the call).
template <typename T>
static inline cudaError_t sdc_malloc(T **p, size_t bytes)
{
    if (bytes == 0) bytes = 1;
    if (sdc_alloc_denied(bytes)) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, bytes);
}

// Stream-ordered scratch of one call: every buffer taken through get() is
// released on the stream (cudaFreeAsync) when the holder goes out of scope,
// on the error paths as on the normal one.
struct SdcScratch {
    cudaStream_t st;
    std::vector<void *> p;
    explicit SdcScratch(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t get(T **ptr, size_t count)
    {
        cudaError_t e = sdc_alloc(ptr, count, st);
        if (e == cudaSuccess) p.push_back((void *)*ptr);
        return e;
    }
    ~SdcScratch() { for (void *q : p) cudaFreeAsync(q, st); }
    SdcScratch(const SdcScratch &) = delete;
    SdcScratch &operator=(const SdcScratch &) = delete;
};

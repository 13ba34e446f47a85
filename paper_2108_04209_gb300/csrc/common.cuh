// Shared device/host helpers of the SuperDC GB300 library (sm_103a, FP64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "superdc.h"

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

// Stream-ordered scratch allocation helpers.
template <typename T>
static inline cudaError_t sdc_alloc(T **p, size_t count, cudaStream_t st)
{
    if (count == 0) count = 1;
    return cudaMallocAsync((void **)p, count * sizeof(T), st);
}

// Index guards of the checked build (nvcc -DSUPERDC_CHECK; build(check=True)
// makes _lib/libsuperdc_check.so).  An index that a kernel reads from device
// data (a near-list entry, a source row of the permutation, a merged
// position) is tested against the extent of the array it selects from before
// use.  A bad index latches SUPERDC_DEV_INDEX in the status word (read back
// by superdc_sync_status / the call's own status check, which then returns
// SUPERDC_ERR_CUDA) and is replaced by 0, so the access stays inside the array
// and nothing traps.  Without the macro SDC_IDX(i, n, word) is (i): the
// default build's code is unchanged.
#pragma once
#include <stdint.h>
#include <type_traits>
#include "superdc.h"

#if !defined(__CUDACC__) && !defined(__host__)
#define __host__
#endif
#if !defined(__CUDACC__) && !defined(__device__)
#define __device__
#endif

namespace sdc_check {

// i if 0 <= i < n, else 0 with SUPERDC_DEV_INDEX latched in *word (when given)
__host__ __device__ inline int64_t guard(int64_t i, int64_t n, int32_t *word)
{
    if (i >= 0 && i < n) return i;
    if (word) {
#if defined(__CUDA_ARCH__)
        atomicOr(word, SUPERDC_DEV_INDEX);
#else
        *word |= SUPERDC_DEV_INDEX;
#endif
    }
    return 0;
}

}  // namespace sdc_check

#ifdef SUPERDC_CHECK
#define SDC_IDX(i, n, word) \
    ((typename std::decay<decltype(i)>::type)sdc_check::guard((int64_t)(i), (int64_t)(n), (word)))
#else
#define SDC_IDX(i, n, word) (i)
#endif

// The triangular FMM with leaf boxes of 32 indices.
#define FMM_BOX 32
#define FMM_NS fmm_b32
#include "fmm_impl.cuh"

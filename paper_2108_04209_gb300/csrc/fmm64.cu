// The triangular FMM with leaf boxes of 64 indices.
#define FMM_BOX 64
#define FMM_NS fmm_b64
#include "fmm_impl.cuh"

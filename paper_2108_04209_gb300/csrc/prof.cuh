// Per-kernel event timing hooks (active only after superdc_profile_enable(1)).
#pragma once
#include <cuda_runtime.h>

bool prof_on();
// Device work counter of a named kernel (events it counts are algorithmic
// operations), or nullptr when profiling is off.
unsigned long long *prof_counter(const char *name);
void prof_begin(cudaStream_t st);
void prof_end(const char *name, cudaStream_t st);

// Wrap one kernel launch: PROF_LAUNCH("secular", st, kernel<<<...>>>(...));
#define PROF_LAUNCH(name, st, ...)  \
    do {                            \
        prof_begin(st);             \
        __VA_ARGS__;                \
        prof_end(name, st);         \
    } while (0)

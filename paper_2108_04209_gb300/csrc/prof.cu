// Optional per-kernel CUDA-event timing (benchmark instrumentation).
#include <cuda_runtime.h>
#include <string.h>
#include <vector>
#include "common.cuh"
#include "prof.cuh"

namespace {
struct Slot {
    const char *name;
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
bool g_on = false;
std::vector<Slot> g_slots;
std::vector<std::pair<const char *, unsigned long long *>> g_ctr;
cudaEvent_t g_open = nullptr;

Slot *find(const char *name, bool create)
{
    for (auto &s : g_slots)
        if (strcmp(s.name, name) == 0) return &s;
    if (!create) return nullptr;
    g_slots.push_back(Slot());
    g_slots.back().name = name;
    return &g_slots.back();
}

void drain(Slot &s)
{
    for (auto &pr : s.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(pr.second) == cudaSuccess &&
            cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) {
            s.ms += t;
            s.launches++;
        }
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    s.pending.clear();
}
}  // namespace

bool prof_on() { return g_on; }

unsigned long long *prof_counter(const char *name)
{
    if (!g_on) return nullptr;
    for (auto &c : g_ctr)
        if (strcmp(c.first, name) == 0) return c.second;
    unsigned long long *p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(unsigned long long)) != cudaSuccess) { cudaFree(p); return nullptr; }
    g_ctr.push_back({name, p});
    return p;
}

void prof_begin(cudaStream_t st)
{
    if (!g_on) return;
    if (cudaEventCreate(&g_open) != cudaSuccess) { g_open = nullptr; return; }
    cudaEventRecord(g_open, st);
}

void prof_end(const char *name, cudaStream_t st)
{
    if (!g_on || !g_open) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    find(name, true)->pending.push_back({g_open, e});
    g_open = nullptr;
}

extern "C" {

superdc_status superdc_profile_enable(int32_t on)
{
    g_on = (on != 0);
    return SUPERDC_OK;
}

superdc_status superdc_profile_reset(void)
{
    for (auto &s : g_slots) {
        drain(s);
        s.launches = 0;
        s.ms = 0.0;
    }
    for (auto &c : g_ctr) cudaMemset(c.second, 0, sizeof(unsigned long long));
    return SUPERDC_OK;
}

superdc_status superdc_profile_counter(const char *name, int64_t *value)
{
    if (!name || !value) return SUPERDC_ERR_ARG;
    for (auto &c : g_ctr) {
        if (strcmp(c.first, name) != 0) continue;
        unsigned long long v = 0;
        if (cudaMemcpy(&v, c.second, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return SUPERDC_ERR_CUDA;
        *value = (int64_t)v;
        return SUPERDC_OK;
    }
    *value = 0;
    return SUPERDC_ERR_ARG;
}

superdc_status superdc_profile_read(const char *name, int64_t *launches, double *ms)
{
    if (!name || !launches || !ms) return SUPERDC_ERR_ARG;
    Slot *s = find(name, false);
    if (!s) { *launches = 0; *ms = 0.0; return SUPERDC_ERR_ARG; }
    drain(*s);
    *launches = s->launches;
    *ms = s->ms;
    return SUPERDC_OK;
}

}  // extern "C"

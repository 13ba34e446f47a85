// FP64 pipe throughput probe: dependent-free DFMA streams and FP64 reciprocal
// throughput, timed with CUDA events.  Prints one JSON line.
// Every thread runs NCH independent fused multiply-add chains; the grid is a
// multiple of the SM count, so the FP64 pipes of all SMs are saturated.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int NCH = 8;

__global__ void k_dfma(double *out, int iters, double a, double b)
{
    double x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < NCH; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < NCH; c++) s += x[c];
    if (s == 12345.678) out[0] = s;   // keep the chains alive
}

__global__ void k_drcp(double *out, int iters)
{
    double x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) x[c] = 1.0 + threadIdx.x * 1e-6 + c * 1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < NCH; c++) x[c] = 1.0 / x[c] + 1e-9;
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < NCH; c++) s += x[c];
    if (s == 12345.678) out[0] = s;
}

int main()
{
    int dev = 0, nsm = 0, clk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    double *out;
    cudaMalloc(&out, 8);
    const int threads = 256, blocks = nsm * 8, iters = 1 << 14;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_fma = 1e30f, best_rcp = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0);
        k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best_fma) best_fma = t;
        cudaEventRecord(e0);
        k_drcp<<<blocks, threads>>>(out, iters / 8);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best_rcp) best_rcp = t;
    }
    double nfma = (double)blocks * threads * iters * NCH;
    double nrcp = (double)blocks * threads * (iters / 8) * NCH;
    double tflops = 2.0 * nfma / (best_fma * 1e-3) / 1e12;
    double rcp_per_s = nrcp / (best_rcp * 1e-3);
    cudaError_t err = cudaGetLastError();
    printf("{\"fp64_tflops\": %.4f, \"dfma_per_clk_per_sm\": %.3f, \"fp64_div_per_s\": %.4e, "
           "\"div_cost_in_dfma\": %.2f, \"sms\": %d, \"clock_attr_mhz\": %.0f, \"ms_fma\": %.3f, \"err\": \"%s\"}\n",
           tflops, (nfma / (best_fma * 1e-3)) / (nsm * clk * 1e3), rcp_per_s,
           (nfma / (best_fma * 1e-3)) / rcp_per_s, nsm, clk / 1e3, best_fma, cudaGetErrorString(err));
    return err == cudaSuccess ? 0 : 1;
}

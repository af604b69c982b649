// Throughput probes for the roofline denominators the driver does not
// measure: FP32 fused multiply-add (scalar and packed f32x2), FP32 min / max
// and three-input min (ALU pipe), and the MUFU ex2 / lg2 approximations.  Each thread runs 8 independent dependency chains so the
// pipes, not latencies, limit the rate; the result is lane-operations per
// second over a grid of (SMs x 8) blocks of 256 threads.
#include <cuda_runtime.h>

#include "wts_common.cuh"

namespace wts {

namespace {

constexpr int kChains = 8;

template <int WHICH>
__global__ void __launch_bounds__(256) probe_kernel(float* out, int iters, float seed)
{
    float v[kChains], w[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) { v[c] = seed + 0.001f * (threadIdx.x + c); w[c] = seed - 0.002f * c; }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (WHICH == 0) v[c] = __fmaf_rn(v[c], 0.999f, 0.0001f);
            if (WHICH == 1) { v[c] = fminf(v[c], w[c]); w[c] = fmaxf(w[c], v[c]); }
            if (WHICH == 2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
            if (WHICH == 3) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
            if (WHICH == 4) {
                unsigned long long p;
                asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(v[c]), "f"(w[c]));
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p) : "l"(0x3f7fbe773f7fbe77ull), "l"(0x38d1b71738d1b717ull));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(v[c]), "=f"(w[c]) : "l"(p));
            }
            if (WHICH == 5) asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(v[c]) : "f"(w[c]), "f"(w[(c + 1) % kChains]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c] + w[c];
    if (s == 12345.678f) out[threadIdx.x] = s;   // keeps the chains alive
}

}  // namespace

int run_probe(int which, double* ops_per_s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8, block = 256, iters = 4096;
    float* out = nullptr;   // never written (the guard value is unreachable)
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        switch (which) {
            case 0: probe_kernel<0><<<grid, block>>>(out, iters, 1.0f); break;
            case 1: probe_kernel<1><<<grid, block>>>(out, iters, 1.0f); break;
            case 2: probe_kernel<2><<<grid, block>>>(out, iters, -1.0f); break;
            case 3: probe_kernel<3><<<grid, block>>>(out, iters, 1.5f); break;
            case 4: probe_kernel<4><<<grid, block>>>(out, iters, 1.0f); break;
            default: probe_kernel<5><<<grid, block>>>(out, iters, 1.0f); break;
        }
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess) return 1;
    const double per_chain = (which == 1 || which == 4) ? 2.0 : 1.0;   // two lane-ops per iteration
    *ops_per_s = (double)grid * block * iters * kChains * per_chain / (best * 1e-3);
    return 0;
}

}  // namespace wts

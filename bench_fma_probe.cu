// bench_fma_probe.cu -- a benchmark helper, not part of libbs: the throughput of the arithmetic pipes the
// velocity kernels run on, measured as chains of dependent fused multiply-adds, several independent chains
// per thread, a grid of 8 CTAs of 256 threads per SM.  The iteration loop is unrolled by 4 so that its
// counter and branch take few issue slots (a plain float32 fma issues one instruction per lane operation, so
// every other instruction shows in the rate).  The float32 rate bounds the far sweep (FMA pipe), the float64
// rate the float64 path and the exact near rule.  bench.py (--workload peaks) compiles it on demand.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;


__global__ void __launch_bounds__(kProbeThreads) fma_f64_kernel(double *out, int iters)
{
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1e-3 * (threadIdx.x + j);
#pragma unroll 4
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], 0.9999999, 1e-9);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) fma_f32_kernel(double *out, int iters)
{
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = 1e-3f * (threadIdx.x + j);
#pragma unroll 4
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = fmaf(a[j], 0.9999999f, 1e-9f);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += a[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

// two float32 lanes per register pair, one fma.rn.f32x2 per pair
__global__ void __launch_bounds__(kProbeThreads) fma_f32x2_kernel(double *out, int iters)
{
    unsigned long long a[8], m, c;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float x = 1e-3f * (threadIdx.x + j), y = x + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[j]) : "f"(x), "f"(y));
    }
    const float m0 = 0.9999999f, c0 = 1e-9f;
    asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(m0));
    asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(c0));
#pragma unroll 4
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(m), "l"(c));
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[j]));
        s += x + y;
    }
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

// kind 0: float64 fma, 1: float32 fma, 2: packed float32x2 fma.  Writes the TFLOP/s (2 flop per lane fma)
// of the second of two timed launches on the current device to *tflops.  Returns 0, 1 (bad kind) or
// 2 (a CUDA call failed).
extern "C" __attribute__((visibility("default"))) int fma_probe_rate(int kind, double *tflops)
{
    if (kind < 0 || kind > 2 || !tflops) return 1;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
    cudaStream_t st = nullptr;
    const int blocks = n_sm * kProbeCtasPerSm;
    const int64_t n = (int64_t)blocks * kProbeThreads;
    double *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&buf, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // lane fmas per thread per iteration, and iterations (about 5-20 ms per launch on a GB300)
    const int chains = kind == 0 ? 8 : 16;
    const int iters = kind == 0 ? 4000 : 40000;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        if (kind == 0)
            fma_f64_kernel<<<blocks, kProbeThreads, 0, st>>>(buf, iters);
        else if (kind == 1)
            fma_f32_kernel<<<blocks, kProbeThreads, 0, st>>>(buf, iters);
        else
            fma_f32x2_kernel<<<blocks, kProbeThreads, 0, st>>>(buf, iters);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess) *tflops = 2.0 * chains * (double)iters * (double)n / (ms * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    return e == cudaSuccess ? 0 : 2;
}


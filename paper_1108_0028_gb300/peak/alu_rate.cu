// Arithmetic-rate probe: the issue rate of plain FP32 FMA, paired FP32 FMA (FFMA2), the MUFU
// reciprocal square root and FP64 FMA on the current GPU.  Each thread runs long chains over
// eight independent accumulators (enough independent work to cover the pipe latencies); the
// result is stored so that nothing is optimised away.  No clock, power or other device setting
// is read or changed.  Used by the benchmark to confirm the FP32 peak it divides by.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kAcc = 8;

__global__ void k_ffma(float *out, int iters, float b, float c) {
    float a[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) a[i] = fmaf(a[i], b, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma2(float *out, int iters, float b, float c) {
    float2 a[kAcc];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += a[i].x + a[i].y;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rsqrt(float *out, int iters, float b, float c) {
    float a[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = 1.0f + (float)(threadIdx.x + i) * b + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) a[i] = rsqrtf(a[i]);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(float *out, int iters, float b, float c) {
    double a[kAcc];
    const double bd = b, cd = c;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kAcc; ++i) a[i] = fma(a[i], bd, cd);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace

extern "C" {

// Runs probe `which` (0 FFMA, 1 FFMA2, 2 MUFU rsqrt, 3 DFMA) once on `blocks` x `threads`
// threads with `iters` iterations, into out (device, blocks * threads floats), and returns the
// kernel time in milliseconds (CUDA events on the legacy default stream), or a negative value
// on a CUDA error.  *ops receives the operation count (FMA = 2 flops; rsqrt = 1).
double alu_rate_run(int which, int blocks, int threads, int iters, float *out, double *ops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    const double nthreads = (double)blocks * threads;
    cudaEventRecord(e0, 0);
    switch (which) {
        case 0: k_ffma<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f); *ops = nthreads * iters * kAcc * 2.0; break;
        case 1: k_ffma2<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f); *ops = nthreads * iters * kAcc * 4.0; break;
        case 2: k_rsqrt<<<blocks, threads>>>(out, iters, 1e-6f, 0.5f); *ops = nthreads * iters * kAcc; break;
        default: k_dfma<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f); *ops = nthreads * iters * kAcc * 2.0; break;
    }
    cudaEventRecord(e1, 0);
    float ms = -1.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? (double)ms : -1.0;
}

}

// kns_peak.cu -- measured throughput ceilings of the pipes the render's kernels lean on (and a
// self-test of the bounded device waits, at the end): FP32 fused
// multiply-add (the FP32 MLPs) and the multi-function unit's ex2 (the softplus of every hidden unit
// costs an ex2 and an lg2).  Each micro-kernel keeps eight independent dependency chains per thread
// on every SM and is timed with CUDA events; the roofline of the render is formed against these.
#include <cuda_runtime.h>

#include "kns_wave.cuh"

namespace kns {

__global__ void __launch_bounds__(256) peak_ffma_kernel(float *sink, int iters) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.f + 1e-3f * (float)(threadIdx.x + j);
    const float b = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 1234.5f) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

__device__ __forceinline__ float ex2_mufu(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(256) peak_mufu_kernel(float *sink, int iters) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5f + 1e-3f * (float)(threadIdx.x & 31) + 0.01f * j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = ex2_mufu(-a[j]);  // stays in [0.5, 1]
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

// Times both micro-kernels (one warm-up launch each, then the best of three); per-second rates of FP32
// FLOP (2 per FMA) and ex2 operations.
cudaError_t measure_peaks(int sm_count, cudaStream_t s, double *ffma_flops, double *mufu_ops) {
    constexpr int kThreads = 256, kBlocksPerSM = 8, kIters = 4096;
    const int blocks = sm_count * kBlocksPerSM;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double work = (double)blocks * kThreads * kIters * 4 * 8;  // chain steps
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (which == 0) peak_ffma_kernel<<<blocks, kThreads, 0, s>>>(sink, kIters);
            else peak_mufu_kernel<<<blocks, kThreads, 0, s>>>(sink, kIters);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        if (e == cudaSuccess && best > 0.f) {
            if (which == 0) *ffma_flops = 2.0 * work / (best * 1e-3);
            else *mufu_ops = work / (best * 1e-3);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return e;
}

// ---------------------------------------------------------------- self-test of the bounded waits
// A wait that nothing satisfies, with a short poll limit: which = 0, the mbarrier wait of a tile (no
// arrival ever comes); which = 1, the persistent trace's grid barrier with block 1 of 2 never arriving.
// The waiting threads give up after `polls` polls and record KNS_ERR_TIMEOUT in the status word, as a
// render's waits do, and the kernel returns.
__global__ void __launch_bounds__(128) selftest_timeout_kernel(WaveCtrl *ctrl, int *status, int which,
                                                               uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_flag;
    if (which == 0) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        const bool ok = mbar_wait(&bar, 0u, polls);  // phase 0 needs one arrival; none is made
        if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(status, 0, (int)6 /* KNS_ERR_TIMEOUT */);
    } else {
        if (blockIdx.x == 1) return;  // this block never reaches the barrier
        unsigned gen = 0;
        if (!grid_sync(ctrl, gen, &s_flag, polls) && threadIdx.x == 0) atomicCAS(status, 0, (int)6);
    }
}

cudaError_t launch_selftest_timeout(WaveCtrl *ctrl, int *status, int which, uint32_t polls, cudaStream_t s) {
    selftest_timeout_kernel<<<which == 0 ? 1 : 2, 128, 0, s>>>(ctrl, status, which, polls);
    return cudaGetLastError();
}

}  // namespace kns

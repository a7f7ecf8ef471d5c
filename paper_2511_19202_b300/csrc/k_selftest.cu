// Device checks and measurements that are library services (the paper has no counterpart).
//
// nvgs_selftest_wait_timeout: exercises the failure path of the bounded device-side waits that the
// tensor-core MLP kernels use on their mbarriers (a library service: the paper has no
// counterpart).  One warp waits on an mbarrier that nothing ever arrives on, with the same helper
// (tc::mbar_wait: lane 0 polls, bounded by an iteration count and by one second of the global
// timer); the wait must give up, the kernel must record it and return, and the context must stay
// usable.  No fault, trap or hang is involved.
#include "nvgs_internal.cuh"
#include "tc_common.cuh"

namespace nvgs {
namespace {

// out[0] = 1 if the wait gave up (0 if it completed: impossible here), out[1] = microseconds
// lane 0 spent waiting.
__global__ void __launch_bounds__(32) k_wait_selftest(uint32_t* __restrict__ out) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const uint64_t t0 = tc::global_ns();
    const bool done = tc::mbar_wait(&bar, 0u);   // nothing arrives on `bar`
    const uint64_t t1 = tc::global_ns();
    if (threadIdx.x == 0) {
        out[0] = done ? 0u : 1u;
        const uint64_t us = (t1 - t0) / 1000u;
        out[1] = us > 0xffffffffull ? 0xffffffffu : (uint32_t)us;
    }
}

// FP32 FMA throughput: every thread runs eight independent chains of fused multiply-adds (enough
// independent work per scheduler to cover the FMA latency); the results feed one conditional
// store so that nothing is optimised away.
constexpr int kFmaChains = 8;
constexpr int kFmaUnroll = 16;
__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ out, int iters, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; c++) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; u++)
#pragma unroll
            for (int c = 0; c < kFmaChains; c++) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kFmaChains; c++) s += x[c];
    if (s == -1.0f) out[blockIdx.x] = s;   // never true for the chosen a, b
}

}  // namespace
}  // namespace nvgs

extern "C" nvgs_status nvgs_measure_fp32_fma(int device, double* tflops) {
    if (!tflops) return NVGS_ERR_INVALID_ARG;
    *tflops = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) return NVGS_ERR_INVALID_ARG;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return NVGS_ERR_CUDA;
    const int blocks = sms * 8, threads = 256, iters = 20000;
    float* d = nullptr;
    if (cudaMalloc(&d, (size_t)blocks * sizeof(float)) != cudaSuccess) return NVGS_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        nvgs::k_fma_peak<<<blocks, threads>>>(d, iters / 10, 0.9999999f, 1e-7f);   // warm-up
        cudaEventRecord(e0);
        nvgs::k_fma_peak<<<blocks, threads>>>(d, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(e1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess || !(ms > 0.0f)) return NVGS_ERR_CUDA;
    const double flops = 2.0 * blocks * threads * (double)iters * nvgs::kFmaUnroll * nvgs::kFmaChains;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return NVGS_OK;
}

extern "C" nvgs_status nvgs_selftest_wait_timeout(int device, double* seconds_waited) {
    if (seconds_waited) *seconds_waited = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) return NVGS_ERR_INVALID_ARG;
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, 8) != cudaSuccess) return NVGS_ERR_CUDA;
    uint32_t h[2] = {0u, 0u};
    cudaError_t e = cudaMemset(d, 0, 8);
    if (e == cudaSuccess) {
        nvgs::k_wait_selftest<<<1, 32>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return NVGS_ERR_CUDA;
    if (seconds_waited) *seconds_waited = h[1] * 1e-6;
    return h[0] == 1u ? NVGS_OK : NVGS_ERR_CUDA;
}

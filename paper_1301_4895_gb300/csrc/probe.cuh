// Benchmark helpers: event timing of the contraction kernels and an FMA
// throughput probe (the measured denominator of the ALU roofline).
#pragma once

#include <cuda_runtime.h>

#include "mixed_common.cuh"

#include <cstdint>
#include <mutex>
#include <vector>

namespace mbc {

struct TimingState {
    std::mutex mu;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};

inline TimingState &timing() {
    static TimingState t;
    return t;
}

// record an event pair around a launch when timing is enabled
struct TimedLaunch {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit TimedLaunch(cudaStream_t st) : s(st) {
        TimingState &t = timing();
        std::lock_guard<std::mutex> g(t.mu);
        if (!t.on) return;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            a = b = nullptr;
            return;
        }
        cudaEventRecord(a, s);
    }
    ~TimedLaunch() {
        if (!a) return;
        cudaEventRecord(b, s);
        TimingState &t = timing();
        std::lock_guard<std::mutex> g(t.mu);
        t.ev.push_back({a, b});
    }
};

// FMA throughput probes (the measured denominators of the ALU roofline).
// The FP64 pipe's rate depends on the operand pattern: chains that repeat
// one multiplier and addend register read back slower than the complex
// multiply-accumulate of the contraction kernels (acc += x * y on separate
// real and imaginary accumulators, x and y changing), which is what the FP64
// probe runs. The FP32 probe runs packed FP32-pair FMA chains (the form the
// mixed kernels issue). Every SM is filled to its occupancy limit with one
// wave of equal blocks.
constexpr int kProbeAcc = 4;  // complex accumulators per thread (FP64 probe)
constexpr int kProbeChains = 16;  // packed pair chains per thread (FP32 probe)

__global__ void k_fma_probe64(double *out, int iters) {
    double re[kProbeAcc], im[kProbeAcc];
    double xr = threadIdx.x * 1e-3, xi = 0.5, yr = 0.999, yi = 1e-3;
#pragma unroll
    for (int i = 0; i < kProbeAcc; ++i) {
        re[i] = i;
        im[i] = -i;
    }
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int i = 0; i < kProbeAcc; ++i) {
                re[i] = __fma_rn(xr, yr, re[i]);
                re[i] = __fma_rn(-xi, yi, re[i]);
                im[i] = __fma_rn(xr, yi, im[i]);
                im[i] = __fma_rn(xi, yr, im[i]);
            }
            xr = __fma_rn(xr, 0.9999999, 1e-9);
        }
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < kProbeAcc; ++i) s += re[i] + im[i];
    if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}
// DFMAs per thread of k_fma_probe64
__host__ __device__ constexpr double probe64_fmas(int iters) { return (4.0 * kProbeAcc + 1.0) * iters; }

__global__ void k_fma_probe32(float *out, int iters) {
    uint64_t a[kProbeChains];
    const uint64_t m = f2_pack(0.999999f, 0.999999f), c = f2_pack(1e-7f, 1e-7f);
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = f2_pack((float)(threadIdx.x + i), (float)i);
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i) a[i] = f2_fma(a[i], m, c);
    }
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s ^= a[i];
    if (s == 12345ull) out[blockIdx.x * blockDim.x + threadIdx.x] = 1.f;  // keeps the chains live
}
// FP32 FMAs per thread of k_fma_probe32 (two per packed instruction)
__host__ __device__ constexpr double probe32_fmas(int iters) { return 2.0 * kProbeChains * iters; }

}  // namespace mbc

// Benchmark helpers: event timing of the contraction kernels and an FMA
// throughput probe (the measured denominator of the ALU roofline).
#pragma once

#include <cuda_runtime.h>

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

// FMA throughput probe: NCH independent multiply-add chains per thread, the
// loop unrolled so that loop control is a small fraction of the issue slots.
// Launched with every SM filled to its occupancy limit (one wave of equal
// blocks), so no SM idles while others finish.
template <class T>
__global__ void k_fma_probe(T *out, int iters, T seed) {
    constexpr int NCH = 16;
    T a[NCH];
#pragma unroll
    for (int i = 0; i < NCH; ++i) a[i] = seed + (T)(threadIdx.x + i);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < NCH; ++i) a[i] = a[i] * m + c;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < NCH; ++i) s += a[i];
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}
constexpr int kProbeChains = 16;

}  // namespace mbc

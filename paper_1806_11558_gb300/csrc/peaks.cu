// peaks.cu -- measured FMA throughput of this GPU (FP64 and FP32), the
// denominators of the ALU rooflines of the entry-evaluation kernels and of
// the FP64 product.  Nominal figures (unit counts x clock) overstate what the
// FP64 pipe of this part delivers, so the roofline fractions are taken
// against a measurement instead.  The paper has no counterpart.
//
// Every thread runs eight independent FMA chains a <- a * b + c for `iters`
// steps (b just below 1, c small, so the values stay bounded); the chains
// give each warp scheduler enough independent instructions to keep its FMA
// pipe busy, and the loop is unrolled 16 steps deep so that its counter and
// branch take ~2 % of the issue slots.  The result is 2 x (threads x 8 x iters) / kernel time.
#include <algorithm>

#include "hm_internal.cuh"

namespace hm {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 16;  // steps per loop iteration: 128 FMAs per 3 loop instructions

template <class T>
__global__ void __launch_bounds__(PK_THREADS) fma_peak_kernel(const T *__restrict__ seed, int iters,
                                                              T *__restrict__ sink) {
    const T b = seed[0], c = seed[1];
    T a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = seed[2] + (T)(threadIdx.x + k);
    for (int i = 0; i < iters; i += PK_UNROLL) {  // iters is a multiple of PK_UNROLL
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    // never true for the seeds used; keeps every chain live
    if (s == seed[3]) sink[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

template <class T> static double measure(int iters, cudaStream_t s) {
    const int sms = num_sms();
    const int blocks = sms * (2048 / PK_THREADS);  // a full SM of threads each
    DBuf seed, sink;
    seed.alloc(sizeof(T) * 4);
    sink.alloc(sizeof(T) * (size_t)blocks * PK_THREADS);
    const T h[4] = {(T)0.9999999, (T)1e-3, (T)0.5, (T)-12345.0};
    HM_CUDA_CHECK(cudaMemcpyAsync(seed.p, h, sizeof(h), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    HM_CUDA_CHECK(cudaEventCreate(&e0));
    HM_CUDA_CHECK(cudaEventCreate(&e1));
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up; the best of the other three counts
        HM_CUDA_CHECK(cudaEventRecord(e0, s));
        fma_peak_kernel<T><<<blocks, PK_THREADS, 0, s>>>(seed.as<T>(), iters, sink.as<T>());
        HM_LAUNCH_CHECK();
        HM_CUDA_CHECK(cudaEventRecord(e1, s));
        HM_CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        HM_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        const double flops = 2.0 * (double)blocks * PK_THREADS * PK_CHAINS * (double)iters;
        if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

double measure_fma_peak(hm_dtype kind, cudaStream_t s) {
    // about 20-40 ms per launch on a GB300 at full clock
    return kind == HM_F64 ? measure<double>(12000, s) : measure<float>(600000, s);  // multiples of 16
}

}  // namespace hm

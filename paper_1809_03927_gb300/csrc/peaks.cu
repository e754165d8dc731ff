// Micro-benchmarks of the two throughputs that bound the transport (Sec. 2.C
// engine): the issue rate of the SM's FP32/INT32 lanes and the rate of
// 64-bit integer atomic additions to L2-resident memory (the dose tally).
// Each kernel runs a fixed, small amount of work (a few milliseconds) on
// every SM; dose_measure_peaks times them with CUDA events.
#include <cuda_runtime.h>
#include <cstdint>

#include "dose.h"
#include "kernels.h"

namespace dose {
namespace {

// kMix: per iteration 8 FFMA, 4 IMAD and 4 LOP3 on independent chains (the
// transport's mix of FP32 arithmetic, 32-bit products and bit logic); else
// 16 FFMA.  Inline PTX keeps each instruction and its count.
template <bool kMix>
__global__ void __launch_bounds__(1024) k_peak_issue(float *out, unsigned *iout, int iters, float m, float c,
                                                    unsigned km, unsigned kc)
{
    float a[8];
    unsigned b[4];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = threadIdx.x * (k + 1);
    // unrolled 16 times: the loop's own counter and branch add about 1 %
#pragma unroll 16
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(m), "f"(c));
        if (kMix) {
#pragma unroll
            for (int k = 0; k < 4; ++k) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(b[k]) : "r"(km), "r"(kc));
#pragma unroll
            for (int k = 0; k < 4; ++k)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(b[k]) : "r"(km), "r"(kc));
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(c), "f"(m));
        }
    }
    float s = 0.0f;
    unsigned t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) t ^= b[k];
    if (s == 12345.678f) out[threadIdx.x] = s;          // keeps the chains live; never true
    if (t == 0x9E3779B9u && kMix) iout[threadIdx.x] = t;
}

// 64-bit atomic additions (reductions: the result is not used, as in the
// tally) to pseudo-random elements of an array of mask + 1 elements.
__global__ void __launch_bounds__(1024) k_peak_red(unsigned long long *a, unsigned mask, int iters)
{
    unsigned x = (blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u + 0x7F4A7C15u;
    for (int it = 0; it < iters; ++it) {
        x ^= x << 13; x ^= x >> 17; x ^= x << 5;       // xorshift32
        atomicAdd(a + (x & mask), 1ull);
    }
}

}  // namespace
}  // namespace dose

using namespace dose;

extern "C" int dose_measure_peaks(double out[4], void *stream)
{
    if (!out) {
        set_thread_error("out is NULL");
        return DOSE_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr unsigned kTallyWords = 1u << 21;          // 16.8 MB: the slab workload's tally
    unsigned long long *arr = nullptr;
    float *fo = nullptr;
    unsigned *io = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&arr, kTallyWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&fo, 1024 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&io, 1024 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(arr, 0, kTallyWords * sizeof(unsigned long long), st);
    const unsigned grid = (unsigned)(2 * sms), block = 1024;   // 64 warps per SM
    const double threads = (double)grid * block;
    // best of three timings of each kernel, after a warm-up launch
    auto timed = [&](auto launch) -> double {
        double best = 1e30;
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) { launch(); e = cudaGetLastError(); }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms > 0.0f && ms < best) best = ms;
        }
        return best * 1e-3;
    };
    const int it_issue = 16384, it_red = 1024;        // about 2 ms and 1 ms
    const double t_mix = timed([&] { k_peak_issue<true><<<grid, block, 0, st>>>(fo, io, it_issue, 1.0000001f, 1e-7f, 2654435761u, 12345u); });
    const double t_fma = timed([&] { k_peak_issue<false><<<grid, block, 0, st>>>(fo, io, it_issue, 1.0000001f, 1e-7f, 2654435761u, 12345u); });
    const double t_red = timed([&] { k_peak_red<<<grid, block, 0, st>>>(arr, kTallyWords - 1, it_red); });
    if (e == cudaSuccess) {
        out[0] = threads * it_issue * 16.0 / t_mix;     // FP32/INT32 thread instructions per second
        out[1] = threads * it_issue * 16.0 / t_fma;     // FFMA thread instructions per second
        out[2] = threads * it_red / t_red;              // 64-bit atomic additions per second
        out[3] = (double)sms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(arr);
    cudaFree(fo);
    cudaFree(io);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return DOSE_ECUDA;
    }
    return DOSE_OK;
}

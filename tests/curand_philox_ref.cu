// Test helper, compiled by tests/test_gpu_curand.py: cuRAND's own
// Philox4_32_10 (device API) at given (seed, subsequence, offset), so the
// engine's generator can be checked against NVIDIA's by calling it.
// curand_init keys the generator with the seed's two 32-bit words, puts the
// subsequence in the counter's upper 64 bits and offset / 4 in its lower 64
// bits; curand4 then returns the 128-bit block at that counter.
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {
__global__ void k_curand_philox(const unsigned long long *seed, const unsigned long long *subsequence,
                                const unsigned long long *offset, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], subsequence[i], offset[i], &st);
    out[i] = curand4(&st);
}
}  // namespace

// Host arrays in and out; returns a cudaError_t.
extern "C" int curand_philox_blocks(const unsigned long long *seed, const unsigned long long *subsequence,
                                    const unsigned long long *offset, unsigned *out_words, int n)
{
    unsigned long long *d = nullptr;
    uint4 *o = nullptr;
    const size_t b = (size_t)n * sizeof(unsigned long long);
    cudaError_t e = cudaMalloc(&d, 3 * b);
    if (e == cudaSuccess) e = cudaMalloc(&o, (size_t)n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(d, seed, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, subsequence, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 2 * n, offset, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_curand_philox<<<(n + 127) / 128, 128>>>(d, d + n, d + 2 * n, o, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_words, o, (size_t)n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d);
    cudaFree(o);
    return (int)e;
}

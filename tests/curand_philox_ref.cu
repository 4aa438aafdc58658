// Test helper: Philox4x32-10 blocks from cuRAND's device API (an implementation
// independent of the oracle), used to pin all four counter words of the oracle's
// generator.  curand_init(seed, subsequence, offset) starts at counter
// (offset/4 as 64 bits in words 0-1, subsequence as 64 bits in words 2-3), key
// (seed low, seed high); with offset % 4 == 0 the first curand4() returns the
// Philox output of that counter.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void blocks_kernel(uint64_t seed, const unsigned long long* subseq, const unsigned long long* offset,
                              int n, uint4* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq[k], offset[k], &st);
    out[k] = curand4(&st);
}

extern "C" int curand_philox_blocks(uint64_t seed, const unsigned long long* subseq,
                                    const unsigned long long* offset, int n, uint32_t* out_host)
{
    unsigned long long *d_s = nullptr, *d_o = nullptr;
    uint4* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_s, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_s, subseq, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_o, offset, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        blocks_kernel<<<(n + 63) / 64, 64>>>(seed, d_s, d_o, n, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_host, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_s);
    cudaFree(d_o);
    cudaFree(d_out);
    return (int)e;
}

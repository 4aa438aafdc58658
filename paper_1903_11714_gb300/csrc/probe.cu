// Integer-pipe throughput probe: the denominator of the sweep's ALU roofline.
//
// The sweep's arithmetic is dominated by Philox's 32x32->64 multiplies and
// three-input XORs.  These kernels run long chains of independent multiplies
// (or XORs) with no memory traffic and report operations per SM per clock,
// measured with clock64 on every resident block.
#include <cstdint>

#include "ising.h"
#include "ising_internal.cuh"

namespace ising {
namespace {

constexpr int kChains = 16;
constexpr int kIters = 4096;

__global__ void mulwide_probe(uint32_t seed, uint32_t* sink, long long* cycles)
{
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + threadIdx.x * 7u + k;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            // one full 32x32->64 product per step, both halves consumed (as in a Philox round)
            const uint64_t p = (uint64_t)0xD2511F53u * a[k];
            a[k] = (uint32_t)(p >> 32) ^ (uint32_t)p;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= a[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void xor3_probe(uint32_t seed, uint32_t* sink, long long* cycles)
{
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + threadIdx.x * 13u + k;
    const uint32_t c1 = seed * 3u + 1u, c2 = seed * 5u + 7u;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __funnelshift_l(a[k], a[k], 1) ^ c1 ^ (c2 + k);
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= a[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace ising

extern "C" int ising_probe_int_rates(double out[2])
{
    using namespace ising;
    if (!out) return ISING_EINVAL;
    const int threads = 512, per_sm = 2;
    const int blocks = sm_count() * per_sm;
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(uint32_t) * blocks * threads) != cudaSuccess) return ISING_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
        cudaFree(sink);
        return ISING_ENOMEM;
    }
    long long* h = new long long[blocks];
    for (int which = 0; which < 2; ++which) {
        for (int rep = 0; rep < 2; ++rep) {  // first run warms clocks and caches
            if (which == 0)
                mulwide_probe<<<blocks, threads>>>(12345u, sink, cyc);
            else
                xor3_probe<<<blocks, threads>>>(12345u, sink, cyc);
        }
        if (cudaMemcpy(h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete[] h;
            cudaFree(sink);
            cudaFree(cyc);
            return ISING_ECUDA;
        }
        long long worst = 1;
        for (int b = 0; b < blocks; ++b) worst = h[b] > worst ? h[b] : worst;
        // per chain step: one 32x32->64 multiply (probe 0) or two ALU ops, a funnel
        // shift and a 3-input XOR (probe 1)
        const double ops = (double)kIters * kChains * threads * per_sm * (which == 0 ? 1.0 : 2.0);
        out[which] = ops / (double)worst;
    }
    delete[] h;
    cudaFree(sink);
    cudaFree(cyc);
    return ISING_OK;
}

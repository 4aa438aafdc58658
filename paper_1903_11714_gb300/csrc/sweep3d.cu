// Three-dimensional checkerboard sweep: launchers of the kernel in sweep3d_kernel.cuh
// (whose header comment describes the method), start states, observables and the
// int8 copy of rows.
#include <cstdint>

#include "ising_internal.cuh"
#include "sweep3d.cuh"
#include "sweep3d_kernel.cuh"

namespace ising {
namespace {

using namespace cubic;

constexpr int kThreads3 = kCubicThreads;

// (M, E) of a state: every bond joins a black and a white site, so counting the
// white sites' six anti-aligned neighbours counts each anti-aligned bond once.
template <int NT, int G>
__global__ void __launch_bounds__(NT) cubic_observe_kernel(const uint32_t* __restrict__ black,
                                                           const uint32_t* __restrict__ white, int64_t L,
                                                           int64_t* ME)
{
    __shared__ unsigned long long red[2 * (NT / 32)];
    const int W = (int)(L / 64), WG = W / G;
    const int64_t ngroups = L * L * WG;
    unsigned long long ups = 0, anti = 0;
    for (int64_t g = (int64_t)blockIdx.x * NT + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * NT) {
        const int64_t r = g / WG;
        const int w = (int)(g - r * WG) * G;
        const int64_t i = r / L, j = r - i * L;
        Nbr<G> n;
        load_neighbours<G>(black, L, W, i, j, w, (int)((i + j + 1) & 1), n);
        uint32_t t[G];
        load_ro<G>(white + r * W + w, t);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            ups += __popc(t[k]) + __popc(n.sm[k]);
            anti += __popc(t[k] ^ n.up[k]) + __popc(t[k] ^ n.dn[k]) + __popc(t[k] ^ n.no[k]) + __popc(t[k] ^ n.so[k]) +
                    __popc(t[k] ^ n.sm[k]) + __popc(t[k] ^ n.hz[k]);
        }
    }
    block_add_twice<NT>(ups, anti, red, ME);
}

__global__ void cubic_set_pair(int64_t* p, int64_t a, int64_t b)
{
    p[0] = a;
    p[1] = b;
}

// Start state: hot = sites whose uniform with sweep slot 0xFFFFFFFF is below 2^31 (~R_0); cold = all +1.
__global__ void cubic_init_kernel(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start)
{
    const int64_t W = L / 64, words = L * L * W;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = idx >= words;
        const int64_t e = idx - c * words;
        uint32_t* plane = c ? white : black;
        if (start == 1) {
            plane[e] = 0xFFFFFFFFu;
            continue;
        }
        // plane word e = r * W + w holds plane indices 32 e .. 32 e + 31
        plane[e] = hot_start_word((uint64_t)e, (uint32_t)c, key);
    }
}

__global__ void cubic_unpack_kernel(const uint32_t* __restrict__ black, const uint32_t* __restrict__ white,
                                    int8_t* lat, int64_t L, int64_t row0, int64_t nrows)
{
    const int64_t W = L / 64;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nrows * W;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = idx / W, w = idx - a * W;
        const int64_t r = row0 + a, i = r / L, j = r - i * L;
        const uint32_t bw[2] = {black[r * W + w], white[r * W + w]};
        int8_t* out = lat + a * L + 64 * w;
        for (int c = 0; c < 2; ++c) {
            const int off = (int)((i + j + c) & 1);
            for (int b = 0; b < 32; ++b) out[2 * b + off] = ((bw[c] >> b) & 1u) ? (int8_t)1 : (int8_t)-1;
        }
    }
}

int grid3(int64_t work, int threads)
{
    const int64_t want = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_cubic_init(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start, cudaStream_t s)
{
    cubic_init_kernel<<<grid3(2 * L * L * (L / 64), 256), 256, 0, s>>>(black, white, L, key, start);
    return cudaGetLastError();
}

cudaError_t launch_cubic_observe(const uint32_t* black, const uint32_t* white, int64_t L, int64_t* ME,
                                 cudaStream_t s)
{
    cubic_set_pair<<<1, 1, 0, s>>>(ME, -L * L * L, -3 * L * L * L);
    const int64_t W = L / 64;
    if (W % 4 == 0)
        cubic_observe_kernel<256, 4><<<grid3(L * L * W / 4, 256), 256, 0, s>>>(black, white, L, ME);
    else
        cubic_observe_kernel<256, 1><<<grid3(L * L * W, 256), 256, 0, s>>>(black, white, L, ME);
    return cudaGetLastError();
}

int cubic_words_per_group(int64_t L) { return (L / 64) % 4 == 0 ? 4 : 1; }

cudaError_t launch_cubic_half_sweep(const CubicDesc& d, unsigned long long* work, int colour, uint32_t sweep,
                                    cudaStream_t s, const void* const* fixed)
{
    const int64_t L = d.L, W = d.W;
    const int G = cubic_words_per_group(L);
    const int64_t groups = L * L * (W / G);
    const int64_t resident = 2 * (int64_t)sm_count();
    const int64_t need = (groups + kThreads3 - 1) / kThreads3;
    const int grid = (int)(need < resident ? need : resident);
    if (fixed && fixed[colour]) {
        // the instance compiled for this lattice's thresholds (jit.cu), same parameters
        CubicDesc dd = d;
        void* args[] = {&dd, &colour, &sweep, &work};
        return cudaLaunchKernel(fixed[colour], dim3(grid), dim3(kThreads3), args, 0, s);
    }
    if (G == 4 && colour == 1)
        cubic_half_sweep_kernel<kThreads3, 4, true><<<grid, kThreads3, 0, s>>>(d, colour, sweep, work);
    else if (G == 4)
        cubic_half_sweep_kernel<kThreads3, 4, false><<<grid, kThreads3, 0, s>>>(d, colour, sweep, work);
    else if (colour == 1)
        cubic_half_sweep_kernel<kThreads3, 1, true><<<grid, kThreads3, 0, s>>>(d, colour, sweep, work);
    else
        cubic_half_sweep_kernel<kThreads3, 1, false><<<grid, kThreads3, 0, s>>>(d, colour, sweep, work);
    return cudaGetLastError();
}

cudaError_t launch_cubic_unpack(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                                int64_t nrows, cudaStream_t s)
{
    cubic_unpack_kernel<<<grid3(nrows * (L / 64), 256), 256, 0, s>>>(black, white, lat, L, row0, nrows);
    return cudaGetLastError();
}

}  // namespace ising

// Bit-packed checkerboard half-sweep: launchers, shared-memory limits and occupancy
// of the kernel in sweep_packed_kernel.cuh (whose header comment describes the
// method), and the per-call sweep-counter advance.
#include "ising_internal.cuh"
#include "jit.h"
#include "sweep_packed_kernel.cuh"

namespace ising {
namespace {

using namespace sweep;

// After `steps` sweeps: advance each live lattice's sweep counter (bounded by its target).
__global__ void packed_advance_kernel(LatticeDesc* desc, const int32_t* count, int steps)
{
    const int n = *count;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        LatticeDesc& d = desc[l];
        if (!d.active) continue;
        const uint64_t nxt = (uint64_t)d.sweep + (uint64_t)steps;
        d.sweep = (uint32_t)(nxt < d.target ? nxt : (uint64_t)(d.sweep < d.target ? d.target : d.sweep));
    }
}

}  // namespace

int packed_smem_header_bytes(int threads)
{
    return 128 + ((2 * (threads / 32) * 4 + 127) / 128) * 128 + (threads / 32) * queue_cap(threads) * 16;
}

template <int NT>
void launch_nt(const TileTable& tt, const LatticeDesc* one, int colour, int step, int* status, int grid, size_t smem,
               int stage_words, cudaStream_t s, long long wait_limit, uint32_t extra_tx, bool blocks)
{
    if (one && one->tile_words != 0 && one->tile_words != one->W)
        packed_half_sweep_kernel<NT, true, 1><<<grid, NT, smem, s>>>(tt, *one, colour, step, status, stage_words,
                                                                     wait_limit, extra_tx);
    else if (one)
        packed_half_sweep_kernel<NT, true, 0><<<grid, NT, smem, s>>>(tt, *one, colour, step, status, stage_words,
                                                                     wait_limit, extra_tx);
    else if (blocks)
        packed_half_sweep_kernel<NT, false, 2><<<grid, NT, smem, s>>>(tt, LatticeDesc{}, colour, step, status,
                                                                      stage_words, wait_limit, extra_tx);
    else
        packed_half_sweep_kernel<NT, false, 0><<<grid, NT, smem, s>>>(tt, LatticeDesc{}, colour, step, status,
                                                                      stage_words, wait_limit, extra_tx);
}

cudaError_t launch_packed_half_sweep(const TileTable& tt, int colour, int step, int* status, int grid, int threads,
                                     int smem_stage_bytes, cudaStream_t s, long long wait_limit, uint32_t extra_tx,
                                     const LatticeDesc* one, bool blocks, const void* fixed)
{
    int stage_words = smem_stage_bytes / 4;
    const size_t smem = (size_t)packed_smem_header_bytes(threads) + 2 * (size_t)smem_stage_bytes;
    if (fixed) {
        // an instance compiled for the thresholds of this lattice (one) or of every lattice
        // of the table (jit.cu): the same parameters as the built-in instances
        TileTable t = tt;
        LatticeDesc d = one ? *one : LatticeDesc{};
        void* args[] = {&t, &d, &colour, &step, &status, &stage_words, &wait_limit, &extra_tx};
        return cudaLaunchKernel(fixed, dim3(grid), dim3(threads), args, smem, s);
    }
    switch (threads) {
    case 128:
        launch_nt<128>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx, blocks);
        break;
    case 256:
        launch_nt<256>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx, blocks);
        break;
    case 512:
        launch_nt<512>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx, blocks);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NT>
cudaError_t set_limit_nt(size_t bytes)
{
    const size_t most = (size_t)packed_smem_header_bytes(NT) + 2 * (size_t)kStageCapBytes;
    if (bytes < most) bytes = most;
    cudaError_t e = cudaFuncSetAttribute(packed_half_sweep_kernel<NT, false, 2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(packed_half_sweep_kernel<NT, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(packed_half_sweep_kernel<NT, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(packed_half_sweep_kernel<NT, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    return e;
}

cudaError_t packed_set_smem_limit(int threads, size_t bytes)
{
    switch (threads) {
    case 128:
        return set_limit_nt<128>(bytes);
    case 256:
        return set_limit_nt<256>(bytes);
    case 512:
        return set_limit_nt<512>(bytes);
    default:
        return cudaErrorInvalidValue;
    }
}

template <int NT>
cudaError_t occupancy_nt(size_t smem, int* blocks_per_sm, bool one)
{
    // the lower of the instance's two builds
    int a = 0, b = 0;
    cudaError_t e = one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, packed_half_sweep_kernel<NT, true, 0>, NT, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, packed_half_sweep_kernel<NT, false, 0>, NT, smem);
    if (e == cudaSuccess)
        e = one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, packed_half_sweep_kernel<NT, true, 1>, NT, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, packed_half_sweep_kernel<NT, false, 2>, NT, smem);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

cudaError_t packed_occupancy(int threads, size_t smem, int* blocks_per_sm, bool one)
{
    switch (threads) {
    case 128:
        return occupancy_nt<128>(smem, blocks_per_sm, one);
    case 256:
        return occupancy_nt<256>(smem, blocks_per_sm, one);
    case 512:
        return occupancy_nt<512>(smem, blocks_per_sm, one);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t packed_fixed_configure(const void* fixed, size_t smem, int threads, int* blocks_per_sm)
{
    size_t bytes = (size_t)packed_smem_header_bytes(threads) + 2 * (size_t)kStageCapBytes;
    if (smem > bytes) bytes = smem;
    cudaError_t e = cudaFuncSetAttribute(fixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fixed, threads, smem);
    return e;
}

cudaError_t launch_packed_advance(LatticeDesc* desc, const int32_t* count, int max_count, int steps, cudaStream_t s)
{
    const int threads = 128;
    const int grid = (max_count + threads - 1) / threads;
    packed_advance_kernel<<<grid > 0 ? grid : 1, threads, 0, s>>>(desc, count, steps);
    return cudaGetLastError();
}

}  // namespace ising

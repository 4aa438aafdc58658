// Launchers of the three-dimensional checkerboard sweep (sweep3d.cu).
//
// The Sec. 3 Hamiltonian on the cubic L x L x L torus (d = 3), with the paper's
// checkerboard rules (Sec. 3.1, Algorithms 1-2) and six neighbours per site.
// Layout: two bit planes (colour c = (i+j+k) & 1), each L*L rows of W = L/64
// words; row r = i*L + j, bit b of word w of row r of plane c is the site
// (i, j, 2(32w+b) + ((i+j+c) & 1)), 1 = +1.  Plane index p = r*(L/2) + 32w + b,
// plane word r*W + w; its uniforms are the 2D ones (philox.cuh): bit b of the 32
// random words of calls q = 8 (r*W + w) + 0..7, counter (sweep, q low, c, q high),
// key = seed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ising_device.cuh"

namespace ising {

cudaError_t launch_cubic_init(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start, cudaStream_t s);
// Start-state (M, E) into ME[0..1].
cudaError_t launch_cubic_observe(const uint32_t* black, const uint32_t* white, int64_t L, int64_t* ME,
                                 cudaStream_t s);
// One half-sweep of colour `colour` of sweep `sweep`; the colour-0 launch opens
// hist[sweep] and the colour-1 launch adds the fused (M, E) counts.  work: the
// lattice's two work counters (device memory, zero before its first half-sweep; the
// launches keep them so).  fixed (may be null): the two colours' instances compiled
// for the lattice's thresholds (jit_cubic_kernels), launched instead of the built-in
// ones.
cudaError_t launch_cubic_half_sweep(const CubicDesc& d, unsigned long long* work, int colour, uint32_t sweep,
                                    cudaStream_t s, const void* const* fixed = nullptr);
// Words per thread group of the 3D sweep for side L (4 when L/64 is a multiple of 4).
int cubic_words_per_group(int64_t L);
constexpr int kCubicThreads = 256;
// int8 copy of rows [row0, row0 + nrows) (row r = i*L + j, L bytes each); `lat`
// points at row row0.
cudaError_t launch_cubic_unpack(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                                int64_t nrows, cudaStream_t s);

}  // namespace ising

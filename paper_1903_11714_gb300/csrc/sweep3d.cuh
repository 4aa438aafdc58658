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

namespace ising {

// One cubic lattice of a half-sweep launch (passed by value).
struct CubicDesc {
    uint32_t* plane[2];        // [0] black, [1] white; each L*L*W words
    int64_t* hist;             // (M, E) pairs indexed by sweep number
    uint64_t key;              // Philox key (seed)
    int32_t L, W;              // side, words per plane row (L / 64)
    uint32_t t2, t4, t6;       // thresholds min(T, 2^32 - 1) for h = 2, 4, 6
    uint32_t all2, all4, all6; // ~0u when the threshold is 2^32
};

constexpr int64_t kCubicMaxL = 8192;

// Cubic sides whose Philox call index q = 8 (p >> 5) stays below 2^32 (so the
// per-launch Philox constants hold for every word).
__host__ __device__ inline bool cubic_q_small(int64_t L) { return (uint64_t)L * L * L <= (1ull << 35); }

cudaError_t launch_cubic_init(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start, cudaStream_t s);
// Start-state (M, E) into ME[0..1].
cudaError_t launch_cubic_observe(const uint32_t* black, const uint32_t* white, int64_t L, int64_t* ME,
                                 cudaStream_t s);
// One half-sweep of colour `colour` of sweep `sweep`; the colour-0 launch opens
// hist[sweep] and the colour-1 launch adds the fused (M, E) counts.
cudaError_t launch_cubic_half_sweep(const CubicDesc& d, int colour, uint32_t sweep, cudaStream_t s);
// int8 copy of rows [row0, row0 + nrows) (row r = i*L + j, L bytes each); `lat`
// points at row row0.
cudaError_t launch_cubic_unpack(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                                int64_t nrows, cudaStream_t s);

}  // namespace ising

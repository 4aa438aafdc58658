// Device-side types and constants of the packed sweep, shared by the library's
// translation units and by the run-time compilation of the sweep kernel for a
// lattice's thresholds (NVRTC, which has no C++ standard library headers).
#pragma once
#if defined(__CUDACC_RTC__)
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#else
#include <cstdint>
#endif

namespace ising {

// Device status word values (written by kernels, read by the host).
enum : int { kStatusOk = 0, kStatusTimeout = 1, kStatusBadTile = 2 };

// One lattice of a packed sweep launch.  Planes hold L rows of W = L/64 32-bit
// words; bit b of word w of row i of plane c is the site (i, 2(32w+b) + ((i+c)&1)),
// bit = 1 meaning spin +1.  Plane index p = i*L/2 + 32w + b (the compact colour
// sub-lattices of Sec. 3.2, bit-packed).
struct LatticeDesc {
    uint32_t* plane[2];   // [0] black (colour 0), [1] white (colour 1)
    int64_t* hist;        // (M, E) pairs indexed by sweep number
    uint64_t key;         // Philox key (seed)
    int32_t L;            // side
    int32_t W;            // words per plane row = L / 64
    uint32_t t2, t4;      // thresholds min(T, 2^32 - 1) for h = 2, 4
    uint32_t all2, all4;  // ~0u when the threshold is 2^32 (accept every word)
    int32_t tile_rows;    // rows per tile (multiple of 4, divides L)
    int32_t halo_rows;    // rows staged above/below a tile: 1 if W % 4 == 0, else 4
    uint32_t sweep;       // index of the next sweep of this lattice
    uint32_t target;      // sweeps stop at this index (serving); 0xFFFFFFFF otherwise
    int32_t active;       // 0: skipped by the kernels
    int32_t tile_words;   // words per tile row: W (whole rows), or a divisor of W that is a
                          // multiple of 4 (W % 4 == 0): column blocks, each source row
                          // staged with 4 halo words on either side
};
static_assert(sizeof(LatticeDesc) % 16 == 0, "descriptor alignment");

// Tile table of a launch: tile_start[l] = first global tile of lattice l,
// tile_start[count] = total tiles; one half-sweep visits every tile once.
struct TileTable {
    const LatticeDesc* desc;
    const int32_t* tile_start;  // count + 1 entries
    const int32_t* count;       // device scalar: number of lattices
};

// Words of one pipeline stage for a lattice's tile: source rows (with halos) then
// target rows.  Whole-row tiles (tile_words == W) stage rows of W words; column
// blocks stage source rows of tile_words + 8 words (4 halo words on either side).
__host__ __device__ inline int64_t stage_words(int32_t W, int32_t tile_rows, int32_t halo_rows,
                                               int32_t tile_words = 0)
{
    if (tile_words == 0 || tile_words == W)
        return (int64_t)(tile_rows + 2 * halo_rows) * W + (int64_t)tile_rows * W;
    return (int64_t)(tile_rows + 2 * halo_rows) * (tile_words + 8) + (int64_t)tile_rows * tile_words;
}

// Tiles of one lattice: row blocks times column blocks.
__host__ __device__ inline int64_t lattice_tiles(int64_t L, int32_t tile_rows, int32_t tile_words)
{
    const int64_t W = L / 64;
    return (L / tile_rows) * (W / (tile_words ? tile_words : W));
}

// Largest shared-memory stage of the tiled sweep (two stages per CTA).
constexpr int64_t kStageCapBytes = 100 * 1024;

// Bound on every mbarrier wait of the sweep kernel, in SM clocks (~2 s at 2 GHz,
// far beyond any tile copy).  After it the kernel records kStatusTimeout and
// its CTAs return.
constexpr long long kWaitLimitCycles = 4000000000LL;

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

}  // namespace ising

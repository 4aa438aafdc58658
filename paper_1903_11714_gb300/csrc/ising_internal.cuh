// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

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

// Launchers (return cudaError_t of the launch).  extra_tx > 0 makes every tile
// barrier expect bytes that never arrive: only the timeout self-test uses it.
// one != nullptr: a launch over that single lattice, whose descriptor (with the
// sweep index the host knows) is passed by value; tt is then not read.  Not for
// graph capture, since the sweep index is baked into the launch.  blocks: some
// lattice of tt may have column-block tiles (tile_words < W).
cudaError_t launch_packed_half_sweep(const TileTable& tt, int colour, int step, int* status, int grid,
                                     int threads, int smem_stage_bytes, cudaStream_t s,
                                     long long wait_limit = kWaitLimitCycles, uint32_t extra_tx = 0,
                                     const LatticeDesc* one = nullptr, bool blocks = false);
// One small lattice (L <= packed_resident_max_L()) swept nsweeps times by a single
// CTA holding both planes in shared memory; writes hist[d.sweep .. +nsweeps).
int packed_resident_max_L();
cudaError_t launch_packed_resident(const LatticeDesc& d, int nsweeps, cudaStream_t s);
cudaError_t launch_packed_advance(LatticeDesc* desc, const int32_t* count, int max_count, int steps,
                                  cudaStream_t s);
cudaError_t launch_packed_init(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start,
                               cudaStream_t s);
cudaError_t launch_packed_observe(const uint32_t* black, const uint32_t* white, int64_t L, int64_t* ME,
                                  cudaStream_t s);
// Layout conversion of rows [row0, row0 + nrows); `lat` points at row row0.
cudaError_t launch_pack(const int8_t* lat, uint32_t* black, uint32_t* white, int64_t L, int64_t row0,
                        int64_t nrows, cudaStream_t s);
cudaError_t launch_unpack(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                          int64_t nrows, cudaStream_t s);

cudaError_t launch_int8_init(int8_t* lat, int64_t L, uint64_t key, int start, cudaStream_t s);
cudaError_t launch_int8_half_sweep(int8_t* lat, int64_t L, uint64_t key, uint32_t t2, uint32_t t4, uint32_t all2,
                                   uint32_t all4, uint32_t sweep, int colour, int64_t* hist_slot,
                                   cudaStream_t s);
cudaError_t launch_int8_observe(const int8_t* lat, int64_t L, int64_t* ME, cudaStream_t s);

// Exact moments over hist[first .. first+count): writes 6 doubles
// (abs_m, m2, m4, e, e2, binder) and the exact sums (see moments.cu).
cudaError_t launch_moments(const int64_t* hist, int64_t first, int64_t count, int64_t N, double* out6,
                           uint64_t* sums, cudaStream_t s);

cudaError_t launch_philox_words(uint64_t key, const uint32_t* ctr4, int64_t n, uint32_t* out, cudaStream_t s);

int sm_count();

// Sets the thread-local message that ising_last_error() returns (api.cu).
void set_last_error(const char* msg);

// Packed sweep kernel configuration helpers (sweep_packed.cu).
int packed_smem_header_bytes(int threads);
// Allows launches with up to max(bytes, header + 2 stages of kStageCapBytes) of dynamic
// shared memory on every instance of the sweep kernel for `threads`.  The limit is
// per kernel, shared by every engine of the process, so it is never set below the
// largest launch any engine can make.
cudaError_t packed_set_smem_limit(int threads, size_t bytes);
// Resident CTAs per SM of the sweep kernel: the single-lattice instance (one) or
// the general one, which the two launch bounds give different register budgets.
cudaError_t packed_occupancy(int threads, size_t smem, int* blocks_per_sm, bool one = false);

}  // namespace ising

// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ising_device.cuh"

namespace ising {

// Launchers (return cudaError_t of the launch).  extra_tx > 0 makes every tile
// barrier expect bytes that never arrive: only the timeout self-test uses it.
// one != nullptr: a launch over that single lattice, whose descriptor (with the
// sweep index the host knows) is passed by value; tt is then not read.  Not for
// graph capture, since the sweep index is baked into the launch.  blocks: some
// lattice of tt may have column-block tiles (tile_words < W).  fixed: an instance
// compiled for the thresholds (jit_sweep_kernel) of that lattice (with one) or of
// every lattice of tt (without), launched instead of the built-in one.
cudaError_t launch_packed_half_sweep(const TileTable& tt, int colour, int step, int* status, int grid,
                                     int threads, int smem_stage_bytes, cudaStream_t s,
                                     long long wait_limit = kWaitLimitCycles, uint32_t extra_tx = 0,
                                     const LatticeDesc* one = nullptr, bool blocks = false,
                                     const void* fixed = nullptr);
// Allows launches of a fixed-threshold kernel with `smem` bytes of dynamic shared
// memory (never less than two full stages) and gives its resident CTAs per SM.
cudaError_t packed_fixed_configure(const void* fixed, size_t smem, int threads, int* blocks_per_sm);
// One small lattice (L <= packed_resident_max_L()) swept nsweeps times by a single
// CTA holding both planes in shared memory; writes hist[d.sweep .. +nsweeps).
int packed_resident_max_L();
cudaError_t launch_packed_resident(const LatticeDesc& d, int nsweeps, cudaStream_t s);
cudaError_t launch_packed_advance(LatticeDesc* desc, const int32_t* count, int max_count, int steps,
                                  cudaStream_t s);
// Cluster-resident sweeps (sweep_cluster.cu): lattices of one side L <= cluster_max_L()
// kept in the shared memory of one thread-block cluster of C CTAs each (threads per
// CTA, dynamic shared memory per CTA).  cluster_plan gives the plan for `count`
// lattices (C = 0: none fits); the launch runs nsweeps sweeps of every live lattice of
// desc[0..count), each stopping at its limit.
struct ClusterPlan {
    int C = 0;
    int threads = 0;
    size_t smem = 0;
};
int cluster_max_L();
ClusterPlan cluster_plan(int64_t L, int count);
cudaError_t launch_cluster_sweeps(const LatticeDesc* desc, int count, int64_t L, const ClusterPlan& p, int nsweeps,
                                  cudaStream_t s);
// Parameter blocks of the by-value updates (each under the 4 KB kernel-parameter limit).
struct TileChunk {
    static constexpr int kMax = 960;
    int32_t first, n, count;  // entries first .. first+n-1; count >= 0: also set the lattice count
    int32_t v[kMax];
};
struct GatherChunk {
    static constexpr int kMax = 960;
    int32_t n;
    int32_t idx[kMax];
};
// Enqueue a descriptor write, a tile-table write (n entries and the lattice count), and
// the (sweeps, M, E) gather of batch slots idx[0..n) into out[3n] (device-accessible);
// none waits for the stream's earlier work and the host arrays may change on return.
cudaError_t launch_set_desc(LatticeDesc* dst, const LatticeDesc& d, cudaStream_t s);
cudaError_t launch_set_tiles(int32_t* tile_start, int32_t* count_dst, const int32_t* v, int32_t n, int32_t count,
                             cudaStream_t s);
cudaError_t launch_gather(const LatticeDesc* desc, const int32_t* idx, int32_t n, int64_t* out, cudaStream_t s);
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

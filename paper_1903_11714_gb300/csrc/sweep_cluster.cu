// Cluster-resident sweep of a batch of small bit-packed lattices.
//
// The checkerboard schedule of Sec. 3.1 needs, per half-sweep, every site of one
// colour updated from the other colour's plane; a small lattice is swept many times
// (the temperature scans of Sec. 4.1).  Here each lattice lives for a whole run in
// the shared memory of one thread-block cluster: CTA r of a cluster of C holds rows
// [r L/C, (r+1) L/C) of both bit planes, plus one halo row above and below each
// plane, which it reads after every half-sweep from the neighbouring CTAs' shared
// memory (distributed shared memory, the torus wrapping round the cluster).  A
// cluster barrier separates half-sweeps; nothing goes to global memory between the
// start of a run and its end except each sweep's (M, E).  Clusters do not wait for
// each other, so every lattice runs its sweeps at its own pace in one launch.
//
// The word update is the tiled kernel's (update_tile in sweep_packed_kernel.cuh:
// the same neighbours, Philox keying by global plane index, bit-plane comparison and
// per-warp queue, and the same fused counts), applied to the CTA's block of rows as
// one tile whose results are written in place (a queued word keeps its old value
// until its drain, which finishes it from that value).  The chain is the tiled
// kernel's, bit for bit.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <tuple>

#include "ising_internal.cuh"
#include "sweep_packed_kernel.cuh"

namespace cg = cooperative_groups;

namespace ising {
namespace {

using namespace sweep;

// Shared memory of one CTA of NT threads: the warps' queues, then the two planes,
// each (rows + 2) rows of W words (row 0 and row rows + 1 are the halo rows).
size_t cluster_smem_bytes(int64_t L, int C, int NT)
{
    const int64_t W = L / 64, rows = L / C;
    return (size_t)(NT / 32) * queue_cap(NT) * 16 + 2 * (size_t)(rows + 2) * W * 4;
}

// A CTA asking for more than half of an SM's shared memory has the SM to itself.
constexpr size_t kSpreadBytes = 116 * 1024;

// Rows `rows` (the last) and 1 (the first) of the neighbouring CTAs' copy of plane p
// into this CTA's halo rows 0 and rows + 1.
__device__ __forceinline__ void refresh_halo(cg::cluster_group& cluster, uint32_t* plane, int rows, int W, int rank,
                                             int C)
{
    const int prev = rank == 0 ? C - 1 : rank - 1, next = rank + 1 == C ? 0 : rank + 1;
    const uint32_t* pp = cluster.map_shared_rank(plane, prev);
    const uint32_t* pn = cluster.map_shared_rank(plane, next);
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        plane[k] = pp[(size_t)rows * W + k];
        plane[(size_t)(rows + 1) * W + k] = pn[(size_t)W + k];
    }
}

// One cluster per lattice of the table (lattice = cluster index); nsweeps sweeps of
// each live lattice, each stopping at its own limit.  G words per thread group as in
// the tiled kernel.
template <int NT, int G>
__global__ void __launch_bounds__(NT) cluster_sweep_kernel(const LatticeDesc* __restrict__ desc, int count,
                                                           int nsweeps)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int lat = (int)(blockIdx.x / C);
    if (lat >= count) return;  // the whole cluster leaves together
    const LatticeDesc d = desc[lat];
    if (!d.active || d.sweep >= d.target) return;
    const uint32_t left = d.target - d.sweep;
    const int n = (uint32_t)nsweeps < left ? nsweeps : (int)left;
    if (n <= 0) return;

    extern __shared__ __align__(16) uint4 smem_c[];
    __shared__ unsigned long long red[2 * (NT / 32)];
    const int W = d.W, L = d.L, rows = L / C, i0 = rank * rows;
    const int tid = threadIdx.x, lane = tid & 31;
    uint4* wq = smem_c + (tid >> 5) * queue_cap(NT);
    // a plane sits at the same offset in every CTA of the cluster, so map_shared_rank of
    // the local pointer finds the neighbour's rows
    uint32_t* pl[2];
    pl[0] = reinterpret_cast<uint32_t*>(smem_c + (NT / 32) * queue_cap(NT));
    pl[1] = pl[0] + (size_t)(rows + 2) * W;

    // own rows of both planes into rows 1 .. rows
    for (int k = tid; k < rows * W; k += NT) {
        pl[0][W + k] = d.plane[0][(size_t)i0 * W + k];
        pl[1][W + k] = d.plane[1][(size_t)i0 * W + k];
    }
    cluster.sync();
    refresh_halo(cluster, pl[0], rows, W, rank, C);
    refresh_halo(cluster, pl[1], rows, W, rank, C);
    __syncthreads();

    const uint64_t N = (uint64_t)L * L;
    for (int s = 0; s < n; ++s) {
        const uint32_t sweep = d.sweep + (uint32_t)s;
        int64_t* slot = d.hist + 2 * (int64_t)sweep;
        for (int colour = 0; colour < 2; ++colour) {
            if (colour == 0 && rank == 0 && tid == 0) {
                // this sweep's (M, E): M = 2 * ups - N, E = 2 * anti - 2N (counts added by the white pass)
                slot[0] = -(int64_t)N;
                slot[1] = -2 * (int64_t)N;
            }
            TileCtx x;
            x.s_src = pl[colour ^ 1];
            x.s_tgt = pl[colour] + W;
            x.out = pl[colour] + W;
            x.q_tile = 8ull * (uint64_t)i0 * (uint64_t)W;
            x.key = d.key;
            x.sweep = sweep;
            x.t2 = d.t2;
            x.t4 = d.t4;
            x.all2 = d.all2;
            x.all4 = d.all4;
            x.zero2 = (d.t2 == 0u && d.all2 == 0u) ? ~0u : 0u;
            x.zero4 = (d.t4 == 0u && d.all4 == 0u) ? ~0u : 0u;
            x.W = W;
            x.HB = 1;
            x.colour = colour;
            x.CW = W;
            x.SW = W;
            x.par0 = (i0 + colour) & 1;
            x.q_small = L <= 131072;
            const PhiloxWordConsts pc = philox_consts(d.key, 0u, sweep, (uint32_t)colour);
            uint32_t ups = 0, anti = 0;
            if (colour == 1)
                update_tile<NT, G, true, false, RuntimeThresholds, true>(x, pc, rows * W, wq, ups, anti);
            else
                update_tile<NT, G, false, false, RuntimeThresholds, true>(x, pc, rows * W, wq, ups, anti);
            if (colour == 1) {
                const uint32_t u = __reduce_add_sync(0xffffffffu, ups);
                const uint32_t a = __reduce_add_sync(0xffffffffu, anti);
                if (lane == 0) {
                    red[2 * (tid >> 5)] = u;
                    red[2 * (tid >> 5) + 1] = a;
                }
                __syncthreads();
                if (tid == 0) {
                    unsigned long long su = 0, sa = 0;
                    for (int k = 0; k < NT / 32; ++k) {
                        su += red[2 * k];
                        sa += red[2 * k + 1];
                    }
                    atomicAdd(reinterpret_cast<unsigned long long*>(slot), 2ull * su);
                    atomicAdd(reinterpret_cast<unsigned long long*>(slot + 1), 2ull * sa);
                }
            }
            // plane `colour` is final in every CTA of the lattice (and the slot's opening
            // precedes every count added to it); its halo rows are the next source's
            cluster.sync();
            if (s + 1 < n || colour == 0) {
                refresh_halo(cluster, pl[colour], rows, W, rank, C);
                __syncthreads();
            }
        }
    }
    // no CTA reads another's shared memory after the last cluster barrier, so each may
    // write back its rows and leave
    for (int k = tid; k < rows * W; k += NT) {
        d.plane[0][(size_t)i0 * W + k] = pl[0][W + k];
        d.plane[1][(size_t)i0 * W + k] = pl[1][W + k];
    }
}

template <int NT, int G>
cudaError_t config_g(const LatticeDesc* desc, int count, int C, int nsweeps, size_t smem, cudaStream_t s,
                     int* clusters)
{
    auto kern = cluster_sweep_kernel<NT, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters ? C : count * C));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (clusters) return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
    return cudaLaunchKernelEx(&cfg, kern, desc, count, nsweeps);
}

int words_per_group(int64_t L)
{
    const int64_t W = L / 64;
    return W % 4 == 0 ? 4 : (W % 2 == 0 ? 2 : 1);
}

// Launch (clusters == nullptr) or residency query (the number of clusters of the plan
// resident at once into *clusters) of the instance for the plan's threads and L's group.
cudaError_t config(const LatticeDesc* desc, int count, int64_t L, const ClusterPlan& p, int nsweeps,
                   cudaStream_t s, int* clusters)
{
    const int G = words_per_group(L);
    if (p.threads == 512) {
        if (G == 4) return config_g<512, 4>(desc, count, p.C, nsweeps, p.smem, s, clusters);
        if (G == 2) return config_g<512, 2>(desc, count, p.C, nsweeps, p.smem, s, clusters);
        return config_g<512, 1>(desc, count, p.C, nsweeps, p.smem, s, clusters);
    }
    if (G == 4) return config_g<256, 4>(desc, count, p.C, nsweeps, p.smem, s, clusters);
    if (G == 2) return config_g<256, 2>(desc, count, p.C, nsweeps, p.smem, s, clusters);
    return config_g<256, 1>(desc, count, p.C, nsweeps, p.smem, s, clusters);
}

// Clusters of the plan resident at once on the current device (0: none), cached.
int resident_clusters(int64_t L, const ClusterPlan& p)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int64_t, int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, L, p.C, p.threads, p.smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int clusters = 0;
    if (p.smem + 1024 <= 227 * 1024) {  // with the static reduction array
        if (config(nullptr, 0, L, p, 0, nullptr, &clusters) != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
    }
    cache[key] = clusters;
    return clusters;
}

}  // namespace

int cluster_max_L() { return 4096; }

ClusterPlan cluster_plan(int64_t L, int count)
{
    ClusterPlan none;
    if (L < 64 || L % 64 || L > cluster_max_L() || count < 1) return none;
    auto valid = [&](int C) { return L % C == 0 && L / C >= 16; };
    // spread: as many CTAs as fit one per SM, each of 512 threads with the SM to
    // itself (the cluster scheduler would otherwise pair CTAs on some SMs and leave
    // others idle), the largest cluster whose clusters are all resident at once
    for (int C = 16; C >= 1; C /= 2) {
        if (!valid(C) || (int64_t)count * C > sm_count()) continue;
        ClusterPlan p{C, 512, std::max(cluster_smem_bytes(L, C, 512), kSpreadBytes)};
        if (resident_clusters(L, p) >= count) return p;
    }
    // packed: 256-thread CTAs, as many per SM as fit, the largest cluster whose clusters
    // are all resident at once; else one CTA per lattice, the lattices in waves
    for (int C = 16; C >= 1; C /= 2) {
        if (!valid(C)) continue;
        ClusterPlan p{C, 256, cluster_smem_bytes(L, C, 256)};
        if (resident_clusters(L, p) >= count) return p;
    }
    ClusterPlan p{1, 256, cluster_smem_bytes(L, 1, 256)};
    if (resident_clusters(L, p) > 0) return p;
    return none;
}

cudaError_t launch_cluster_sweeps(const LatticeDesc* desc, int count, int64_t L, const ClusterPlan& p, int nsweeps,
                                  cudaStream_t s)
{
    return config(desc, count, L, p, nsweeps, s, nullptr);
}

}  // namespace ising

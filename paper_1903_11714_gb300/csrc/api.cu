// C ABI (include/ising.h): single-lattice handles, batches, checkpoints, the
// tile autotuner and device building blocks.  Host code only; every step of the
// sweep runs in the kernels of sweep_packed.cu, sweep_int8.cu, lattice_ops.cu
// and moments.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ising.h"
#include "arena.h"
#include "ising_internal.cuh"
#include "jit.h"
#include "sweep3d.cuh"

using namespace ising;

namespace {

thread_local std::string t_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ISING_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(ISING_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// Largest packed side (2^40 sites, 128 GB of planes).  Rows too long for a whole-row
// tile (W = L/64 > 4264) are cut into column blocks, which needs W % 4 == 0 (see
// packed_L_ok).
constexpr int64_t kPackedMaxL = 1 << 20;
constexpr int64_t kInt8MaxL = 1 << 17;
constexpr uint32_t kNoTarget = 0xFFFFFFFFu;
constexpr int64_t kMaxSweeps = 0xFFFFFFFEll;  // sweep counter is a 32-bit Philox counter word

// Handle kind of a cubic (3D) lattice; the public kernel ids are ISING_PACKED
// and ISING_INT8 (2D).
constexpr int kKernelCubic = 2;

// Kernels compiled for a lattice's thresholds (jit.cu): process-wide mode, and the
// smallest side the automatic mode specialises (a compile of a few seconds is then
// repaid within some thousands of sweeps).
std::atomic<int> g_specialize{ISING_SPECIALIZE_AUTO};
constexpr int64_t kSpecializeMinL = 16384;

// Acceptance thresholds T_h = min(2^32, ceil(exp(-2 beta h) 2^32)), h = 2, 4
// (and h = 6 when n = 3, for the cubic lattice).
bool thresholds(double beta, uint64_t* T, int n = 2)
{
    if (!std::isfinite(beta) || beta < 0.0) return false;
    for (int k = 0; k < n; ++k) {
        const double p = std::exp(-2.0 * beta * (double)(2 * (k + 1)));
        double t = std::ceil(p * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        T[k] = (uint64_t)t;
    }
    return true;
}

void set_thresholds(LatticeDesc& d, const uint64_t T[2])
{
    d.t2 = T[0] >= 4294967296ull ? 0xFFFFFFFFu : (uint32_t)T[0];
    d.t4 = T[1] >= 4294967296ull ? 0xFFFFFFFFu : (uint32_t)T[1];
    d.all2 = T[0] >= 4294967296ull ? 0xFFFFFFFFu : 0u;
    d.all4 = T[1] >= 4294967296ull ? 0xFFFFFFFFu : 0u;
}

int halo_rows_for(int64_t W) { return (W % 4 == 0) ? 1 : 4; }

int64_t stage_bytes_for(int64_t L, int tile_rows, int tile_words = 0)
{
    const int64_t W = L / 64;
    const int64_t words = stage_words((int32_t)W, tile_rows, halo_rows_for(W), tile_words);
    return (words * 4 + 15) / 16 * 16;
}

// Tile heights: powers of two from 4 to 256 rows; 2 rows only when a row is a
// whole number of 16-byte units (W % 4 == 0), so that every bulk copy stays
// 16-byte aligned.
constexpr int kMaxTileRows = 256;

bool tile_rows_ok(int64_t L, int tr)
{
    const bool pow2 = tr >= 2 && tr <= kMaxTileRows && (tr & (tr - 1)) == 0;
    return pow2 && (tr >= 4 || (L / 64) % 4 == 0) && tr <= L && L % tr == 0 &&
           stage_bytes_for(L, tr) <= kStageCapBytes;
}

// Column blocks: tile_words = cw < W words of each of tile_rows rows, staged with 4 halo
// words on either side; cw a multiple of 4 dividing W (so W % 4 == 0 and halo rows are
// single rows), below 2^16 (queue entries hold a word's place in 16 bits).
bool tile_ok(int64_t L, int tr, int cw)
{
    const int64_t W = L / 64;
    if (cw == 0 || cw == W) return tile_rows_ok(L, tr);
    const bool pow2 = tr >= 2 && tr <= kMaxTileRows && (tr & (tr - 1)) == 0;
    return pow2 && W % 4 == 0 && cw >= 4 && cw % 4 == 0 && cw < W && W % cw == 0 && cw < 65536 && L % tr == 0 &&
           stage_bytes_for(L, tr, cw) <= kStageCapBytes;
}

// Whole rows fit some tile height.
bool whole_rows_ok(int64_t L)
{
    for (int tr = 2; tr <= kMaxTileRows; tr <<= 1)
        if (tile_rows_ok(L, tr)) return true;
    return false;
}

// Column width of a lattice whose rows are too long for whole-row tiles: the largest
// divisor of W that is a multiple of 4 and at most kBlockWords (2-row blocks of 1,024
// words then take 25 KB per stage, so two CTAs fit an SM); W when whole rows fit; 0
// when neither can be had (W % 4 != 0).
constexpr int kBlockWords = 1024;
int default_tile_words(int64_t L)
{
    const int64_t W = L / 64;
    if (whole_rows_ok(L)) return (int)W;
    if (W % 4) return 0;
    for (int64_t cw = std::min<int64_t>(W - 4, kBlockWords) / 4 * 4; cw >= 4; cw -= 4)
        if (W % cw == 0 && tile_ok(L, 2, (int)cw)) return (int)cw;
    return 0;
}

// A packed side the tiled kernel can sweep: L % 64 == 0, 64 <= L <= 2^20, and a tile
// of some shape fits a stage -- any such L when L % 256 == 0 (whole rows up to
// L = 272,896, column blocks beyond), else L <= 102,336 (whole rows: 4-row tiles with
// 4-row halos).
bool packed_L_ok(int64_t L)
{
    if (L < 64 || L % 64 || L > kPackedMaxL) return false;
    return default_tile_words(L) != 0;
}

// Built-in tile height: about ISING_TILE_WORDS words per tile and at most 64 rows.
// Taller tiles (up to 256 rows) suit big batches and are what ising_autotune picks
// for them, but a batch of a few small lattices cut that way holds fewer tiles than
// the persistent grid has CTAs, so the built-in choice stays short.
#ifndef ISING_TILE_WORDS
#define ISING_TILE_WORDS 4096
#endif
int default_tile_rows(int64_t L, int threads = 256)
{
    const int64_t W = L / 64;
    // lattices of 16,384 and more: 16 words per thread of the CTA (8,192 with 512
    // threads), as for a single handle, so every warp has ~512 words of a tile
    const int64_t words = L >= 16384 ? std::max<int64_t>(ISING_TILE_WORDS, 16 * threads) : ISING_TILE_WORDS;
    int tr = 64;
    while (tr > 2 && ((int64_t)tr * W > words || !tile_rows_ok(L, tr))) tr >>= 1;
    if (!tile_rows_ok(L, tr)) tr = 4;
    return tr;
}

// Tile height for a lattice swept on its own (the single-lattice instance, two
// CTAs per SM): the built-in height, lowered so that small lattices are cut into
// enough tiles to spread over the persistent grid instead of a few large ones.
int single_tile_rows(int64_t L)
{
    const int grid = 2 * sm_count();
    int tr = 4;
    while (tr < kMaxTileRows && L / tr > grid) tr *= 2;
    tr = std::min(tr, default_tile_rows(L));
    while (tr > 2 && !tile_rows_ok(L, tr)) tr >>= 1;
    return tile_rows_ok(L, tr) ? tr : default_tile_rows(L);
}

// CTA size and tile height of a lattice swept on its own.  Sides of at least 16,384
// with whole-row tiles take one 512-thread CTA per SM and tiles of up to 8,192 words,
// so that each of its 16 warps still handles about 512 words of a tile: the per-tile
// costs (the last partial drain of each warp's queue, the stage handoff) are then a
// smaller share than with two 256-thread CTAs of 4,096-word tiles (+2 % at L = 65,536;
// 512-thread CTAs with 4,096-word tiles lose 6 %).  Other sides: 256 threads and
// single_tile_rows.
void single_config(int64_t L, int* tile_rows, int* threads)
{
    *threads = 256;
    *tile_rows = single_tile_rows(L);
    const int64_t W = L / 64;
    if (L < 16384 || !whole_rows_ok(L)) return;
    int best = 0;
    for (int tr = 2; tr <= kMaxTileRows; tr *= 2)
        if (tile_rows_ok(L, tr) && W * tr <= 8192 && L / tr >= 2 * sm_count()) best = tr;
    if (best && W * best >= 4096) {
        *threads = 512;
        *tile_rows = best;
    }
}

// ---------------------------------------------------------------- engine
// The launch state of the packed persistent kernel: descriptor array, tile
// table, status word, grid, and an optional captured graph of k sweeps.
struct Engine {
    cudaStream_t stream = nullptr;
    int threads = 256;
    int grid = 0;
    int stage_bytes = 0;
    int max_count = 0;
    LatticeDesc* d_desc = nullptr;
    int32_t* d_tile_start = nullptr;
    int32_t* d_count = nullptr;
    int* d_status = nullptr;
    std::map<int, cudaGraphExec_t> graphs;  // captured graphs of k sweeps, by k
    // single-lattice handles: host copy of the descriptor, whose sweep field the
    // handle keeps equal to the device's; plain launches then pass it by value
    const LatticeDesc* one = nullptr;
    bool capturing = false;
    bool one_lattice = false;  // launches the single-lattice instance (sizes the grid by its occupancy)
    // single-lattice handles: the instance compiled for the lattice's thresholds (jit.cu),
    // used for the by-value launches; nullptr: the built-in instance
    const void* fixed = nullptr;
    // batches: the multi-lattice instance compiled for the thresholds every lattice of the
    // batch shares, or nullptr (the built-in instance)
    const void* fixed_multi = nullptr;
    // batches of lattices of one side L <= 4096: CTAs per cluster of the cluster-resident
    // sweep (0: the tiled kernel), the side and the table's lattice count
    ClusterPlan cluster;
    int64_t cluster_L = 0;
    int cluster_count = 0;
    bool blocks = false;       // some lattice has column-block tiles (launch the build that handles them)

    void allow_blocks()
    {
        if (!blocks) drop_graph();  // a captured graph holds the whole-row build
        blocks = true;
    }

    int setup(int max_count_, int stage_bytes_, int threads_, cudaStream_t s, bool one_lattice_ = false,
              const void* fixed_ = nullptr)
    {
        one_lattice = one_lattice_;
        fixed = fixed_;
        max_count = max_count_;
        stage_bytes = (stage_bytes_ + 15) / 16 * 16;
        threads = threads_;
        stream = s;
        CK(cudaMalloc(&d_desc, sizeof(LatticeDesc) * (size_t)max_count));
        CK(cudaMalloc(&d_tile_start, sizeof(int32_t) * (size_t)(max_count + 1)));
        CK(cudaMalloc(&d_count, sizeof(int32_t)));
        CK(cudaMalloc(&d_status, sizeof(int)));
        CK(cudaMemsetAsync(d_desc, 0, sizeof(LatticeDesc) * (size_t)max_count, stream));
        CK(cudaMemsetAsync(d_tile_start, 0, sizeof(int32_t) * (size_t)(max_count + 1), stream));
        CK(cudaMemsetAsync(d_count, 0, sizeof(int32_t), stream));
        CK(cudaMemsetAsync(d_status, 0, sizeof(int), stream));
        return configure();
    }

    int configure()
    {
        const size_t smem = (size_t)packed_smem_header_bytes(threads) + 2 * (size_t)stage_bytes;
        CK(packed_set_smem_limit(threads, smem));
        int per_sm = 0;
        CK(packed_occupancy(threads, smem, &per_sm, one_lattice));
        if (fixed || fixed_multi) {
            // the grid follows the instance the launches use
            int per_sm_fixed = 0;
            CK(packed_fixed_configure(fixed ? fixed : fixed_multi, smem, threads, &per_sm_fixed));
            per_sm = per_sm_fixed;
        }
        if (per_sm < 1) return fail(ISING_EINVAL, "sweep kernel does not fit: %d threads, %zu B smem", threads, smem);
        grid = per_sm * sm_count();
        drop_graph();
        return ISING_OK;
    }

    void drop_graph()
    {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }

    // Descriptor and tile-table updates go by value in small kernels, ordered on the
    // stream without waiting for its earlier work (a serving loop admits lattices while
    // earlier sweeps run); tables too long for a few launches are copied and waited for.
    int upload_desc(int idx, const LatticeDesc& d)
    {
        CK(launch_set_desc(d_desc + idx, d, stream));
        return ISING_OK;
    }

    int upload_tiles(const std::vector<int32_t>& tile_start, int32_t count)
    {
        if (tile_start.size() <= 8 * (size_t)TileChunk::kMax) {
            CK(launch_set_tiles(d_tile_start, d_count, tile_start.data(), (int32_t)tile_start.size(), count, stream));
            return ISING_OK;
        }
        CK(cudaMemcpyAsync(d_tile_start, tile_start.data(), sizeof(int32_t) * tile_start.size(),
                           cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(d_count, &count, sizeof(int32_t), cudaMemcpyHostToDevice, stream));
        // pageable source: make sure the driver has consumed it before the vector changes
        CK(cudaStreamSynchronize(stream));
        return ISING_OK;
    }

    TileTable table() const
    {
        TileTable tt;
        tt.desc = d_desc;
        tt.tile_start = d_tile_start;
        tt.count = d_count;
        return tt;
    }

    int enqueue_sweeps(int64_t n)
    {
        const TileTable tt = table();
        const LatticeDesc* by_value = capturing ? nullptr : one;
        for (int64_t k = 0; k < n; ++k) {
            for (int c = 0; c < 2; ++c) {
                cudaError_t e = launch_packed_half_sweep(tt, c, (int)k, d_status, grid, threads, stage_bytes, stream,
                                                         kWaitLimitCycles, 0u, by_value, blocks,
                                                         by_value ? fixed : fixed_multi);
                if (e != cudaSuccess) return cuda_fail(e, "packed half-sweep launch");
            }
        }
        cudaError_t e = launch_packed_advance(d_desc, d_count, max_count, (int)n, stream);
        if (e != cudaSuccess) return cuda_fail(e, "advance launch");
        return ISING_OK;
    }

    int run(int64_t sweeps, int graph_sweeps)
    {
        if (sweeps == 0) return ISING_OK;
        if (cluster.C > 0) {
            // every lattice stays in its cluster's shared memory for up to 4,096 sweeps per
            // launch; no graph is needed
            for (int64_t done = 0; done < sweeps;) {
                const int chunk = (int)std::min<int64_t>(sweeps - done, 4096);
                CK(launch_cluster_sweeps(d_desc, cluster_count, cluster_L, cluster, chunk, stream));
                cudaError_t e = launch_packed_advance(d_desc, d_count, max_count, chunk, stream);
                if (e != cudaSuccess) return cuda_fail(e, "advance launch");
                done += chunk;
            }
            return ISING_OK;
        }
        if (graph_sweeps <= 0) return enqueue_sweeps(sweeps);
        if (sweeps % graph_sweeps) return fail(ISING_EINVAL, "sweeps %lld not a multiple of graph_sweeps %d",
                                               (long long)sweeps, graph_sweeps);
        auto it = graphs.find(graph_sweeps);
        if (it == graphs.end()) {
            if (graphs.size() >= 8) drop_graph();  // a few quantum sizes are kept
            CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            capturing = true;
            int rc = enqueue_sweeps(graph_sweeps);
            capturing = false;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(stream, &g);
            if (rc != ISING_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            it = graphs.emplace(graph_sweeps, ge).first;
        }
        for (int64_t r = 0; r < sweeps / graph_sweeps; ++r) CK(cudaGraphLaunch(it->second, stream));
        return ISING_OK;
    }

    int check_status()
    {
        int st = 0;
        CK(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        if (st != kStatusOk) {
            CK(cudaMemsetAsync(d_status, 0, sizeof(int), stream));
            return fail(ISING_ETIMEOUT, "sweep kernel reported status %d (bounded wait expired)", st);
        }
        return ISING_OK;
    }

    void destroy()
    {
        drop_graph();
        cudaFree(d_desc);
        cudaFree(d_tile_start);
        cudaFree(d_count);
        cudaFree(d_status);
        d_desc = nullptr;
        d_tile_start = nullptr;
        d_count = nullptr;
        d_status = nullptr;
    }
};

int make_stream(void* user, cudaStream_t* s, bool* own)
{
    if (user) {
        *s = (cudaStream_t)user;
        *own = false;
        return ISING_OK;
    }
    CK(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
    *own = true;
    return ISING_OK;
}

// ---------------------------------------------------------------- arena
// First-fit sub-allocator over one device region: the batch's HBM budget.  The
// offsets are kept by FreeList (arena.h); this adds the region.
struct Arena : FreeList {
    char* base = nullptr;

    int init(int64_t bytes)
    {
        reset(bytes);
        CK(cudaMalloc(&base, (size_t)size));
        return ISING_OK;
    }
    void destroy()
    {
        cudaFree(base);
        base = nullptr;
    }
};

}  // namespace

void ising::set_last_error(const char* msg) { t_error = msg; }

// ====================================================================== handles
struct ising_s {
    int64_t L = 0;
    double beta = 0;
    uint64_t seed = 0;
    int start = 0;
    int kernel = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t T[3] = {0, 0, 0};
    Engine eng;          // packed
    LatticeDesc desc{};  // host mirror (packed)
    uint32_t* planes = nullptr;
    int8_t* lat = nullptr;  // int8
    int64_t* hist = nullptr;
    int64_t hist_cap = 0;
    int64_t sweeps_done = 0;
    int64_t* d_me0 = nullptr;   // start-state (M, E)
    unsigned long long* d_work3 = nullptr;  // 3D: the half-sweeps' work counters (one per colour)
    double* d_mom = nullptr;    // 6 doubles
    uint64_t* d_sums = nullptr; // 11 limbs
    std::string kernel_note;    // which sweep kernel runs, and why (ising_specialized)
    const void* cubic_fixed[2] = {nullptr, nullptr};  // 3D: the colours' compiled instances
};

struct ising_batch_s {
    struct Slot {
        bool used = false;
        int64_t L = 0;
        int64_t off = 0, bytes = 0;
        int64_t sweeps_cap = 0;
        int64_t* own_hist = nullptr;  // growable batches: the history, outside the arena
        int64_t done = 0;             // growable batches: sweeps enqueued since admission
        LatticeDesc desc{};
    };
    // growable (made from arrays): lattices have no sweep limit, their histories are
    // allocated apart from the arena and doubled when a run needs more room
    bool growable = false;
    int cluster_mode = ISING_CLUSTER_AUTO;  // ising_batch_set_cluster
    int capacity = 0;
    int64_t max_L = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Engine eng;
    Arena arena;
    std::vector<Slot> slots;
    int32_t count = 0;
    int64_t* d_me = nullptr;
    double* d_mom = nullptr;
    uint64_t* d_sums = nullptr;
};

namespace {

int ensure_hist(ising_t h, int64_t need)
{
    if (need <= h->hist_cap) return ISING_OK;
    int64_t cap = h->hist_cap ? h->hist_cap : 1024;
    while (cap < need) cap *= 2;
    int64_t* nh = nullptr;
    CK(cudaMalloc(&nh, sizeof(int64_t) * 2 * (size_t)cap));
    if (h->hist && h->sweeps_done)
        CK(cudaMemcpyAsync(nh, h->hist, sizeof(int64_t) * 2 * (size_t)h->sweeps_done, cudaMemcpyDeviceToDevice,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(h->hist);
    h->hist = nh;
    h->hist_cap = cap;
    if (h->kernel == ISING_PACKED) {
        h->desc.hist = nh;
        h->desc.sweep = (uint32_t)h->sweeps_done;
        int rc = h->eng.upload_desc(0, h->desc);
        if (rc) return rc;
    }
    return ISING_OK;
}

int check_handle(ising_t h)
{
    if (!h) return fail(ISING_EINVAL, "null handle");
    return ISING_OK;
}

// Words of one colour plane: L rows (2D) or L*L rows (3D) of L/64 words.
int64_t plane_words(ising_t h)
{
    return (h->kernel == kKernelCubic ? h->L * h->L : h->L) * (h->L / 64);
}

// Sites of the lattice: L^2 or L^3.
int64_t site_count(ising_t h) { return (h->kernel == kKernelCubic ? h->L : 1) * h->L * h->L; }

uint32_t thr32(uint64_t T) { return T >= 4294967296ull ? 0xFFFFFFFFu : (uint32_t)T; }
uint32_t all32(uint64_t T) { return T >= 4294967296ull ? 0xFFFFFFFFu : 0u; }

CubicDesc cubic_desc(ising_t h)
{
    CubicDesc d{};
    d.plane[0] = h->planes;
    d.plane[1] = h->planes + plane_words(h);
    d.hist = h->hist;
    d.key = h->seed;
    d.L = (int32_t)h->L;
    d.W = (int32_t)(h->L / 64);
    d.t2 = thr32(h->T[0]);
    d.t4 = thr32(h->T[1]);
    d.t6 = thr32(h->T[2]);
    d.all2 = all32(h->T[0]);
    d.all4 = all32(h->T[1]);
    d.all6 = all32(h->T[2]);
    return d;
}

// int8 copy of a cubic lattice, index (i*L + j)*L + k, through a bounded staging buffer.
// Rows [row0, row0 + nrows) (row r = i*L + j, L sites each) of a cube into out.
int cubic_rows_to_host(ising_t h, int64_t row0, int64_t nrows, int8_t* out)
{
    const int64_t L = h->L;
    const int64_t chunk = std::min<int64_t>(nrows, std::max<int64_t>(1, (int64_t)(256ll << 20) / L));
    int8_t* tmp = nullptr;
    CK(cudaMalloc(&tmp, (size_t)(chunk * L)));
    for (int64_t r0 = 0; r0 < nrows; r0 += chunk) {
        const int64_t nr = std::min<int64_t>(chunk, nrows - r0);
        cudaError_t e =
            launch_cubic_unpack(h->planes, h->planes + plane_words(h), tmp, L, row0 + r0, nr, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out + r0 * L, tmp, (size_t)(nr * L), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(e, "cubic unpack to host");
        }
    }
    cudaFree(tmp);
    return ISING_OK;
}

int cubic_to_host(ising_t h, int8_t* out) { return cubic_rows_to_host(h, 0, h->L * h->L, out); }

int read_status(ising_t h)
{
    if (h->kernel == ISING_PACKED) return h->eng.check_status();
    CK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

// Copies the lattice to host int8 through a bounded device staging buffer.
// Rows [row0, row0 + nrows) of a packed lattice as int8 spins into out (nrows * L bytes).
int packed_rows_to_host(const uint32_t* black, const uint32_t* white, int64_t L, int64_t row0, int64_t nrows,
                        int8_t* out, cudaStream_t s)
{
    const int64_t rows_per = std::max<int64_t>(1, (int64_t)(256ll << 20) / L);
    const int64_t chunk_rows = std::min<int64_t>(nrows, rows_per);
    int8_t* tmp = nullptr;
    CK(cudaMalloc(&tmp, (size_t)(chunk_rows * L)));
    for (int64_t r0 = 0; r0 < nrows; r0 += chunk_rows) {
        const int64_t nr = std::min<int64_t>(chunk_rows, nrows - r0);
        cudaError_t e = launch_unpack(black, white, tmp, L, row0 + r0, nr, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out + r0 * L, tmp, (size_t)(nr * L), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(e, "unpack to host");
        }
    }
    cudaFree(tmp);
    return ISING_OK;
}

int packed_to_host(const uint32_t* black, const uint32_t* white, int64_t L, int8_t* out, cudaStream_t s)
{
    return packed_rows_to_host(black, white, L, 0, L, out, s);
}

int host_to_packed(const int8_t* in, uint32_t* black, uint32_t* white, int64_t L, cudaStream_t s)
{
    const int64_t rows_per = std::max<int64_t>(1, (int64_t)(256ll << 20) / L);
    const int64_t chunk_rows = std::min<int64_t>(L, rows_per);
    int8_t* tmp = nullptr;
    CK(cudaMalloc(&tmp, (size_t)(chunk_rows * L)));
    for (int64_t r0 = 0; r0 < L; r0 += chunk_rows) {
        const int64_t nr = std::min<int64_t>(chunk_rows, L - r0);
        cudaError_t e = cudaMemcpyAsync(tmp, in + r0 * L, (size_t)(nr * L), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_pack(tmp, black, white, L, r0, nr, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(e, "pack from host");
        }
    }
    cudaFree(tmp);
    return ISING_OK;
}

bool spins_valid(const int8_t* in, int64_t n)
{
    for (int64_t k = 0; k < n; ++k)
        if (in[k] != 1 && in[k] != -1) return false;
    return true;
}

int refresh_me0(ising_t h)
{
    cudaError_t e;
    if (h->kernel == kKernelCubic)
        e = launch_cubic_observe(h->planes, h->planes + plane_words(h), h->L, h->d_me0, h->stream);
    else if (h->kernel == ISING_PACKED)
        e = launch_packed_observe(h->planes, h->planes + h->L * (h->L / 64), h->L, h->d_me0, h->stream);
    else
        e = launch_int8_observe(h->lat, h->L, h->d_me0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "observe launch");
    return ISING_OK;
}

void destroy_handle(ising_t h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->eng.destroy();
    cudaFree(h->planes);
    cudaFree(h->lat);
    cudaFree(h->hist);
    cudaFree(h->d_me0);
    cudaFree(h->d_work3);
    cudaFree(h->d_mom);
    cudaFree(h->d_sums);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace

extern "C" {

const char* ising_last_error(void) { return t_error.c_str(); }

const char* ising_version(void) { return "ising-gb300 0.1 (sm_103a)"; }

int ising_thresholds(double beta, uint64_t T[2])
{
    if (!T) return fail(ISING_EINVAL, "null output");
    uint64_t t[2];
    if (!thresholds(beta, t)) return fail(ISING_EINVAL, "beta must be finite and >= 0");
    T[0] = t[0];
    T[1] = t[1];
    return ISING_OK;
}

int ising_init_ex(ising_t* out, int64_t L, double beta, uint64_t seed, int start, int kernel, void* stream)
{
    if (!out) return fail(ISING_EINVAL, "null output");
    uint64_t T[2];
    if (!thresholds(beta, T)) return fail(ISING_EINVAL, "beta must be finite and >= 0");
    if (start != ISING_HOT && start != ISING_COLD) return fail(ISING_EINVAL, "start must be ISING_HOT or ISING_COLD");
    if (kernel == ISING_PACKED) {
        if (!packed_L_ok(L))
            return fail(ISING_EINVAL,
                        "packed kernel needs L %% 64 == 0, 64 <= L, and L <= 272896 (L %% 256 == 0) or L <= 102336");
    } else if (kernel == ISING_INT8) {
        if (L < 8 || L % 8 || L > kInt8MaxL)
            return fail(ISING_EINVAL, "int8 kernel needs L %% 8 == 0 and 8 <= L <= %lld", (long long)kInt8MaxL);
    } else {
        return fail(ISING_EINVAL, "kernel must be ISING_PACKED or ISING_INT8");
    }
    ising_t h = new ising_s();
    h->L = L;
    h->beta = beta;
    h->seed = seed;
    h->start = start;
    h->kernel = kernel;
    h->T[0] = T[0];
    h->T[1] = T[1];
    int rc = make_stream(stream, &h->stream, &h->own_stream);
    if (rc) {
        delete h;
        return rc;
    }
#define CKH(call)                                 \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) {                  \
            int r_ = cuda_fail(e_, #call);        \
            destroy_handle(h);                    \
            return r_;                            \
        }                                         \
    } while (0)
    CKH(cudaMalloc(&h->d_me0, 2 * sizeof(int64_t)));
    CKH(cudaMalloc(&h->d_mom, 6 * sizeof(double)));
    CKH(cudaMalloc(&h->d_sums, 11 * sizeof(uint64_t)));
    if (kernel == ISING_PACKED) {
        const int64_t plane_words = L * (L / 64);
        CKH(cudaMalloc(&h->planes, sizeof(uint32_t) * 2 * (size_t)plane_words));
        CKH(launch_packed_init(h->planes, h->planes + plane_words, L, seed, start, h->stream));
        // whole rows when they fit a tile, else 2-row column blocks
        const int cw = default_tile_words(L);
        int tr = 2, threads = 256;
        if (cw == (int)(L / 64)) single_config(L, &tr, &threads);
        LatticeDesc& d = h->desc;
        d.plane[0] = h->planes;
        d.plane[1] = h->planes + plane_words;
        d.hist = nullptr;
        d.key = seed;
        d.L = (int32_t)L;
        d.W = (int32_t)(L / 64);
        set_thresholds(d, T);
        d.tile_rows = tr;
        d.halo_rows = halo_rows_for(L / 64);
        d.tile_words = cw;
        d.sweep = 0;
        d.target = kNoTarget;
        d.active = 1;
        // the sweep kernel: the resident one for small sides, else the tiled one, compiled
        // for this lattice's thresholds where the mode asks for it and it can be had
        const void* fixed = nullptr;
        const int mode = g_specialize.load();
        if (L <= packed_resident_max_L()) {
            h->kernel_note = "built-in: single-CTA resident kernel (L <= 256)";
        } else if (mode == ISING_SPECIALIZE_OFF) {
            h->kernel_note = "built-in: specialisation switched off";
        } else if (mode == ISING_SPECIALIZE_AUTO && L < kSpecializeMinL) {
            h->kernel_note = "built-in: L below 16384 (automatic mode)";
        } else {
            std::string why;
            fixed = jit_sweep_kernel(threads, cw != (int)(L / 64), d.t2, d.t4, d.all2, d.all4, &why);
            h->kernel_note = fixed ? "specialised: compiled for this lattice's thresholds" : "built-in: " + why;
        }
        rc = h->eng.setup(1, (int)stage_bytes_for(L, tr, cw), threads, h->stream, true, fixed);
        if (rc) {
            destroy_handle(h);
            return rc;
        }
        h->eng.one = &h->desc;
        if (cw != (int)(L / 64)) h->eng.allow_blocks();
        std::vector<int32_t> ts = {0, (int32_t)lattice_tiles(L, tr, cw)};
        rc = h->eng.upload_tiles(ts, 1);
        if (!rc) rc = ensure_hist(h, 1024);
        if (rc) {
            destroy_handle(h);
            return rc;
        }
    } else {
        CKH(cudaMalloc(&h->lat, (size_t)(L * L)));
        CKH(launch_int8_init(h->lat, L, seed, start, h->stream));
        rc = ensure_hist(h, 1024);
        if (rc) {
            destroy_handle(h);
            return rc;
        }
    }
#undef CKH
    rc = refresh_me0(h);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "init");
    }
    if (rc) {
        destroy_handle(h);
        return rc;
    }
    *out = h;
    return ISING_OK;
}

int ising_set_specialize(int32_t mode)
{
    if (mode != ISING_SPECIALIZE_OFF && mode != ISING_SPECIALIZE_AUTO && mode != ISING_SPECIALIZE_ALWAYS)
        return fail(ISING_EINVAL, "mode must be ISING_SPECIALIZE_OFF, _AUTO or _ALWAYS");
    g_specialize.store(mode);
    return ISING_OK;
}

int ising_specialized(ising_t h, int32_t* specialized, char* note, int64_t len)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (specialized) *specialized = (h->eng.fixed || h->cubic_fixed[0]) ? 1 : 0;
    if (note && len > 0) {
        const std::string& n = h->kernel_note.empty() ? std::string("built-in") : h->kernel_note;
        const size_t k = std::min<size_t>(n.size(), (size_t)len - 1);
        memcpy(note, n.data(), k);
        note[k] = '\0';
    }
    return ISING_OK;
}

int ising_init(ising_t* out, int64_t L, double beta, uint64_t seed)
{
    return ising_init_ex(out, L, beta, seed, ISING_HOT, ISING_PACKED, nullptr);
}

int ising_thresholds3d(double beta, uint64_t T[3])
{
    if (!T) return fail(ISING_EINVAL, "null output");
    uint64_t t[3];
    if (!thresholds(beta, t, 3)) return fail(ISING_EINVAL, "beta must be finite and >= 0");
    for (int k = 0; k < 3; ++k) T[k] = t[k];
    return ISING_OK;
}

int ising_init3d(ising_t* out, int64_t L, double beta, uint64_t seed, int start, void* stream)
{
    if (!out) return fail(ISING_EINVAL, "null output");
    uint64_t T[3];
    if (!thresholds(beta, T, 3)) return fail(ISING_EINVAL, "beta must be finite and >= 0");
    if (start != ISING_HOT && start != ISING_COLD) return fail(ISING_EINVAL, "start must be ISING_HOT or ISING_COLD");
    if (L < 64 || L % 64 || L > kCubicMaxL)
        return fail(ISING_EINVAL, "3D lattices need L %% 64 == 0 and 64 <= L <= %lld", (long long)kCubicMaxL);
    ising_t h = new ising_s();
    h->L = L;
    h->beta = beta;
    h->seed = seed;
    h->start = start;
    h->kernel = kKernelCubic;
    for (int k = 0; k < 3; ++k) h->T[k] = T[k];
    int rc = make_stream(stream, &h->stream, &h->own_stream);
    if (rc) {
        delete h;
        return rc;
    }
    // the sweep kernel: compiled for this lattice's thresholds where the mode asks for it
    // (automatic: at least 16384^2 sites) and it can be had, else the built-in one
    const int mode = g_specialize.load();
    if (mode == ISING_SPECIALIZE_OFF) {
        h->kernel_note = "built-in: specialisation switched off";
    } else if (mode == ISING_SPECIALIZE_AUTO && L * L * L < kSpecializeMinL * kSpecializeMinL) {
        h->kernel_note = "built-in: fewer than 16384^2 sites (automatic mode)";
    } else {
        uint32_t t[3], all[3];
        for (int k = 0; k < 3; ++k) {
            t[k] = thr32(T[k]);
            all[k] = all32(T[k]);
        }
        std::string why;
        if (jit_cubic_kernels(kCubicThreads, cubic_words_per_group(L), t, all, h->cubic_fixed, &why))
            h->kernel_note = "specialised: compiled for this lattice's thresholds";
        else
            h->kernel_note = "built-in: " + why;
    }
    cudaError_t e = cudaMalloc(&h->d_me0, 2 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_mom, 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_sums, 11 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->planes, sizeof(uint32_t) * 2 * (size_t)plane_words(h));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_work3, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_work3, 0, 2 * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = launch_cubic_init(h->planes, h->planes + plane_words(h), L, seed, start, h->stream);
    rc = (e == cudaSuccess) ? ensure_hist(h, 1024) : cuda_fail(e, "3D lattice set-up");
    if (!rc) rc = refresh_me0(h);
    if (!rc) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "3D init");
    }
    if (rc) {
        destroy_handle(h);
        return rc;
    }
    *out = h;
    return ISING_OK;
}

int ising_sweep(ising_t h, int64_t n)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (n < 0) return fail(ISING_EINVAL, "n must be >= 0");
    if (n > kMaxSweeps - h->sweeps_done) return fail(ISING_EINVAL, "sweep counter would pass 2^32 - 2");
    if (n == 0) return ISING_OK;
    rc = ensure_hist(h, h->sweeps_done + n);
    if (rc) return rc;
    if (h->kernel == ISING_PACKED && h->L <= packed_resident_max_L()) {
        // small lattice: one CTA keeps both planes on chip for many sweeps per launch
        LatticeDesc d = h->desc;
        for (int64_t done = 0; done < n;) {
            const int64_t chunk = std::min<int64_t>(n - done, 4096);
            d.sweep = (uint32_t)(h->sweeps_done + done);
            cudaError_t e = launch_packed_resident(d, (int)chunk, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "resident sweep launch");
            done += chunk;
        }
    } else if (h->kernel == ISING_PACKED) {
        rc = h->eng.run(n, 0);
        if (rc) return rc;
    } else if (h->kernel == kKernelCubic) {
        const CubicDesc d = cubic_desc(h);
        for (int64_t k = 0; k < n; ++k)
            for (int c = 0; c < 2; ++c) {
                cudaError_t e = launch_cubic_half_sweep(d, h->d_work3, c, (uint32_t)(h->sweeps_done + k), h->stream,
                                                        h->cubic_fixed[0] ? h->cubic_fixed : nullptr);
                if (e != cudaSuccess) return cuda_fail(e, "3D half-sweep launch");
            }
    } else {
        uint32_t t2, t4, all2, all4;
        LatticeDesc tmp{};
        set_thresholds(tmp, h->T);
        t2 = tmp.t2;
        t4 = tmp.t4;
        all2 = tmp.all2;
        all4 = tmp.all4;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t s = h->sweeps_done + k;
            for (int c = 0; c < 2; ++c) {
                cudaError_t e = launch_int8_half_sweep(h->lat, h->L, h->seed, t2, t4, all2, all4, (uint32_t)s, c,
                                                       h->hist + 2 * s, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "int8 half-sweep launch");
            }
        }
    }
    h->sweeps_done += n;
    h->desc.sweep = (uint32_t)h->sweeps_done;
    return ISING_OK;
}

int ising_synchronize(ising_t h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    return read_status(h);
}

int ising_observables(ising_t h, int64_t* M, int64_t* E, int64_t* sweeps_done)
{
    int rc = check_handle(h);
    if (rc) return rc;
    int64_t me[2];
    const int64_t* src = h->sweeps_done ? h->hist + 2 * (h->sweeps_done - 1) : h->d_me0;
    CK(cudaMemcpyAsync(me, src, sizeof(me), cudaMemcpyDeviceToHost, h->stream));
    rc = read_status(h);
    if (rc) return rc;
    if (M) *M = me[0];
    if (E) *E = me[1];
    if (sweeps_done) *sweeps_done = h->sweeps_done;
    return ISING_OK;
}

int ising_history(ising_t h, int64_t first, int64_t count, int64_t* M, int64_t* E)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (first < 0 || count < 0 || first > h->sweeps_done || count > h->sweeps_done - first)
        return fail(ISING_EINVAL, "history range [%lld, %lld) beyond %lld sweeps", (long long)first,
                    (long long)(first + count), (long long)h->sweeps_done);
    std::vector<int64_t> buf(2 * (size_t)count);
    if (count) CK(cudaMemcpyAsync(buf.data(), h->hist + 2 * first, sizeof(int64_t) * buf.size(),
                                  cudaMemcpyDeviceToHost, h->stream));
    rc = read_status(h);
    if (rc) return rc;
    for (int64_t k = 0; k < count; ++k) {
        if (M) M[k] = buf[2 * k];
        if (E) E[k] = buf[2 * k + 1];
    }
    return ISING_OK;
}

int ising_moments_ex(ising_t h, int64_t burn_in, double out[6], uint64_t sums[11])
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(ISING_EINVAL, "null output");
    if (burn_in < 0 || burn_in >= h->sweeps_done) return fail(ISING_EINVAL, "no samples after burn-in");
    CK(launch_moments(h->hist, burn_in, h->sweeps_done - burn_in, site_count(h), h->d_mom, h->d_sums, h->stream));
    double m[6];
    uint64_t s[11];
    CK(cudaMemcpyAsync(m, h->d_mom, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(s, h->d_sums, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    rc = read_status(h);
    if (rc) return rc;
    memcpy(out, m, sizeof(m));
    if (sums) memcpy(sums, s, sizeof(s));
    return ISING_OK;
}

int ising_moments(ising_t h, int64_t burn_in, double* abs_m, double* m2, double* m4, double* e, double* binder)
{
    double m[6];
    int rc = ising_moments_ex(h, burn_in, m, nullptr);
    if (rc) return rc;
    if (abs_m) *abs_m = m[0];
    if (m2) *m2 = m[1];
    if (m4) *m4 = m[2];
    if (e) *e = m[3];
    if (binder) *binder = m[5];
    return ISING_OK;
}

int ising_get_lattice(ising_t h, int8_t* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(ISING_EINVAL, "null output");
    rc = read_status(h);
    if (rc) return rc;
    if (h->kernel == kKernelCubic) return cubic_to_host(h, out);
    if (h->kernel == ISING_PACKED)
        return packed_to_host(h->planes, h->planes + h->L * (h->L / 64), h->L, out, h->stream);
    CK(cudaMemcpyAsync(out, h->lat, (size_t)(h->L * h->L), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_get_rows(ising_t h, int64_t row0, int64_t nrows, int8_t* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out && nrows > 0) return fail(ISING_EINVAL, "null output");
    const int64_t L = h->L, rows = h->kernel == kKernelCubic ? L * L : L;
    if (row0 < 0 || nrows < 0 || nrows > rows - row0)
        return fail(ISING_EINVAL, "rows %lld .. %lld outside 0 .. %lld", (long long)row0, (long long)(row0 + nrows),
                    (long long)rows);
    if (nrows == 0) return ISING_OK;
    rc = read_status(h);
    if (rc) return rc;
    if (h->kernel == kKernelCubic) return cubic_rows_to_host(h, row0, nrows, out);
    if (h->kernel == ISING_PACKED)
        return packed_rows_to_host(h->planes, h->planes + L * (L / 64), L, row0, nrows, out, h->stream);
    CK(cudaMemcpyAsync(out, h->lat + row0 * L, (size_t)(nrows * L), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_set_lattice(ising_t h, const int8_t* in)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!in) return fail(ISING_EINVAL, "null input");
    if (h->kernel == kKernelCubic) return fail(ISING_EINVAL, "set_lattice is for 2D lattices; use set_planes");
    if (!spins_valid(in, h->L * h->L)) return fail(ISING_EINVAL, "lattice entries must be +1 or -1");
    rc = read_status(h);
    if (rc) return rc;
    if (h->kernel == ISING_PACKED) {
        rc = host_to_packed(in, h->planes, h->planes + h->L * (h->L / 64), h->L, h->stream);
        if (rc) return rc;
    } else {
        CK(cudaMemcpyAsync(h->lat, in, (size_t)(h->L * h->L), cudaMemcpyHostToDevice, h->stream));
    }
    if (h->sweeps_done == 0) {
        rc = refresh_me0(h);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_get_planes(ising_t h, uint32_t* black, uint32_t* white)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->kernel == ISING_INT8) return fail(ISING_EINVAL, "not a packed handle");
    const size_t bytes = sizeof(uint32_t) * (size_t)plane_words(h);
    if (black) CK(cudaMemcpyAsync(black, h->planes, bytes, cudaMemcpyDeviceToHost, h->stream));
    if (white) CK(cudaMemcpyAsync(white, h->planes + plane_words(h), bytes, cudaMemcpyDeviceToHost, h->stream));
    return read_status(h);
}

int ising_set_planes(ising_t h, const uint32_t* black, const uint32_t* white)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->kernel == ISING_INT8) return fail(ISING_EINVAL, "not a packed handle");
    if (!black || !white) return fail(ISING_EINVAL, "null input");
    const size_t bytes = sizeof(uint32_t) * (size_t)plane_words(h);
    CK(cudaMemcpyAsync(h->planes, black, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->planes + plane_words(h), white, bytes, cudaMemcpyHostToDevice, h->stream));
    if (h->sweeps_done == 0) {
        rc = refresh_me0(h);
        if (rc) return rc;
    }
    return read_status(h);
}

// ---------------------------------------------------------------- checkpoint
namespace {
struct CkptHeader {
    char magic[8];
    int64_t version, L, kernel, start, sweeps_done, lattice_bytes;
    double beta;
    uint64_t seed;
};
int64_t lattice_bytes(ising_t h)
{
    return h->kernel == ISING_INT8 ? h->L * h->L : (int64_t)sizeof(uint32_t) * 2 * plane_words(h);
}
}  // namespace

int ising_state_bytes(ising_t h, int64_t* bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!bytes) return fail(ISING_EINVAL, "null output");
    *bytes = (int64_t)sizeof(CkptHeader) + lattice_bytes(h) + 16 * h->sweeps_done + 16;
    return ISING_OK;
}

int ising_save(ising_t h, void* buf, int64_t bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    int64_t need = 0;
    ising_state_bytes(h, &need);
    if (!buf || bytes < need) return fail(ISING_EINVAL, "checkpoint buffer needs %lld bytes", (long long)need);
    rc = read_status(h);
    if (rc) return rc;
    CkptHeader hd{};
    memcpy(hd.magic, "ISINGCK1", 8);
    hd.version = 1;
    hd.L = h->L;
    hd.kernel = h->kernel;
    hd.start = h->start;
    hd.sweeps_done = h->sweeps_done;
    hd.lattice_bytes = lattice_bytes(h);
    hd.beta = h->beta;
    hd.seed = h->seed;
    char* p = (char*)buf;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const void* src = h->kernel == ISING_INT8 ? (const void*)h->lat : (const void*)h->planes;
    CK(cudaMemcpyAsync(p, src, (size_t)hd.lattice_bytes, cudaMemcpyDeviceToHost, h->stream));
    p += hd.lattice_bytes;
    CK(cudaMemcpyAsync(p, h->d_me0, 16, cudaMemcpyDeviceToHost, h->stream));
    p += 16;
    if (h->sweeps_done)
        CK(cudaMemcpyAsync(p, h->hist, (size_t)(16 * h->sweeps_done), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_load(ising_t* out, const void* buf, int64_t bytes, void* stream)
{
    if (!out || !buf || bytes < (int64_t)sizeof(CkptHeader)) return fail(ISING_EINVAL, "bad checkpoint buffer");
    CkptHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "ISINGCK1", 8) != 0 || hd.version != 1) return fail(ISING_EINVAL, "not a checkpoint");
    // header fields checked before any device work, so that a damaged blob can
    // neither allocate nor size a copy past the end of buf (16 * sweeps_done and
    // lattice_bytes stay far below 2^63 once these hold)
    if (hd.kernel != ISING_PACKED && hd.kernel != ISING_INT8 && hd.kernel != kKernelCubic)
        return fail(ISING_EINVAL, "checkpoint kernel out of range");
    if (hd.start != ISING_HOT && hd.start != ISING_COLD) return fail(ISING_EINVAL, "checkpoint start out of range");
    if (hd.sweeps_done < 0 || hd.sweeps_done > kMaxSweeps)
        return fail(ISING_EINVAL, "checkpoint sweep count out of range");
    if (hd.lattice_bytes < 0 || hd.lattice_bytes > bytes - (int64_t)sizeof(CkptHeader))
        return fail(ISING_EINVAL, "checkpoint truncated");
    ising_t h = nullptr;
    int rc = hd.kernel == kKernelCubic ? ising_init3d(&h, hd.L, hd.beta, hd.seed, ISING_COLD, stream)
                                       : ising_init_ex(&h, hd.L, hd.beta, hd.seed, ISING_COLD, (int)hd.kernel, stream);
    if (rc) return rc;
    h->start = (int)hd.start;
    if (hd.lattice_bytes != lattice_bytes(h) ||
        bytes < (int64_t)sizeof(CkptHeader) + hd.lattice_bytes + 16 + 16 * hd.sweeps_done) {
        ising_free(h);
        return fail(ISING_EINVAL, "checkpoint truncated");
    }
    const char* p = (const char*)buf + sizeof(CkptHeader);
    void* dst = h->kernel == ISING_INT8 ? (void*)h->lat : (void*)h->planes;
    rc = ensure_hist(h, hd.sweeps_done + 1);
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpyAsync(dst, p, (size_t)hd.lattice_bytes, cudaMemcpyHostToDevice, h->stream);
    p += hd.lattice_bytes;
    if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(h->d_me0, p, 16, cudaMemcpyHostToDevice, h->stream);
    p += 16;
    if (!rc && e == cudaSuccess && hd.sweeps_done)
        e = cudaMemcpyAsync(h->hist, p, (size_t)(16 * hd.sweeps_done), cudaMemcpyHostToDevice, h->stream);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "checkpoint upload");
    if (!rc) {
        h->sweeps_done = hd.sweeps_done;
        h->desc.sweep = (uint32_t)hd.sweeps_done;
        if (h->kernel == ISING_PACKED) rc = h->eng.upload_desc(0, h->desc);
    }
    if (rc) {
        ising_free(h);
        return rc;
    }
    *out = h;
    return ISING_OK;
}

int ising_free(ising_t h)
{
    destroy_handle(h);
    return ISING_OK;
}

// ======================================================================= batch
namespace {
// A batch whose lattices all have one threshold pair sweeps with the multi-lattice
// instance compiled for it (where the mode allows: always, or automatically once the
// batch holds at least 16,384^2 sites); a lattice of another temperature, or a mode
// that forbids it, brings back the built-in instance.  The kernel of captured graphs
// changes with it, so they are dropped and the grid is sized for the new instance.
int update_specialisation(ising_batch_t b)
{
    const int mode = g_specialize.load();
    const LatticeDesc* first = nullptr;
    bool same = true;
    int64_t sites = 0;
    for (const auto& s : b->slots) {
        if (!s.used) continue;
        sites += s.L * s.L;
        if (!first)
            first = &s.desc;
        else if (s.desc.t2 != first->t2 || s.desc.t4 != first->t4 || s.desc.all2 != first->all2 ||
                 s.desc.all4 != first->all4)
            same = false;
    }
    const void* want = nullptr;
    if (first && same && mode != ISING_SPECIALIZE_OFF &&
        (mode == ISING_SPECIALIZE_ALWAYS || sites >= kSpecializeMinL * kSpecializeMinL))
        want = jit_sweep_kernel(b->eng.threads, b->eng.blocks, first->t2, first->t4, first->all2, first->all4, nullptr,
                                false);
    if (want == b->eng.fixed_multi) return ISING_OK;
    b->eng.fixed_multi = want;
    return b->eng.configure();  // drops the graphs and sizes the grid
}

// Lattices of one side L <= 4096 with whole-row tiles are swept by the cluster-resident
// kernel (one thread-block cluster per lattice, all of a run's sweeps in one launch)
// when a cluster plan exists and (in the automatic mode) its estimated rate beats the
// tiled kernel's; otherwise, or when switched off, by the tiled kernel, which spreads
// a few lattices over every SM.  Estimates (GB300 measurements): the cluster form
// sweeps about 22 sites/ns per SM its CTAs occupy (a 512-thread CTA a whole SM, a
// 256-thread one half); the tiled kernel about 25.7 sites/ns per SM at large sizes,
// half of that at 5e7 sites per sweep, below which launch latency dominates.
int update_cluster(ising_batch_t b)
{
    int64_t L = 0;
    bool one_side = true;
    for (const auto& s : b->slots) {
        if (!s.used) continue;
        if (L == 0) L = s.L;
        if (s.L != L || s.desc.tile_words != s.desc.W) one_side = false;
    }
    ClusterPlan p;
    if (b->cluster_mode != ISING_CLUSTER_OFF && L > 0 && one_side && L <= cluster_max_L()) {
        p = cluster_plan(L, b->count);
        if (b->cluster_mode == ISING_CLUSTER_AUTO && p.C > 0) {
            int live = 0;
            for (const auto& s : b->slots) live += s.used && s.desc.active ? 1 : 0;
            const double sms = sm_count(), sites = (double)L * (double)L * live;
            const double used = std::min(sms, (double)b->count * p.C * p.threads / 512.0);
            if (22.0 * used < 25.7 * sms * sites / (sites + 5e7)) p = ClusterPlan();
        }
    }
    b->eng.cluster = p;
    b->eng.cluster_L = L;
    b->eng.cluster_count = b->count;
    return ISING_OK;
}

int rebuild_tiles(ising_batch_t b)
{
    int32_t count = 0;
    for (int k = 0; k < b->capacity; ++k)
        if (b->slots[k].used) count = k + 1;
    std::vector<int32_t> ts((size_t)count + 1, 0);
    for (int k = 0; k < count; ++k) {
        const auto& s = b->slots[k];
        ts[k + 1] = ts[k] + (s.used ? (int32_t)lattice_tiles(s.L, s.desc.tile_rows, s.desc.tile_words) : 0);
    }
    b->count = count;
    int rc = b->eng.upload_tiles(ts, count);
    if (!rc) rc = update_specialisation(b);
    if (!rc) rc = update_cluster(b);
    return rc;
}

// Growable batches: before `sweeps` more sweeps, give every lattice's history room
// for them (doubling; the entries so far are copied).  The kernels read the history
// pointer from the device descriptor, so a captured graph stays valid.
int grow_histories(ising_batch_t b, int64_t sweeps)
{
    for (int k = 0; k < b->capacity; ++k) {
        auto& s = b->slots[k];
        if (!s.used || s.done + sweeps <= s.sweeps_cap) continue;
        int64_t cap = s.sweeps_cap;
        while (cap < s.done + sweeps) cap = std::min<int64_t>(2 * cap, kMaxSweeps + 1);
        int64_t* nh = nullptr;
        CK(cudaMalloc(&nh, 16 * (size_t)cap));
        cudaError_t e = cudaSuccess;
        if (s.done) e = cudaMemcpyAsync(nh, s.own_hist, 16 * (size_t)s.done, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            cudaFree(nh);
            return cuda_fail(e, "history copy");
        }
        cudaFree(s.own_hist);
        s.own_hist = nh;
        s.sweeps_cap = cap;
        s.desc.hist = nh;
        s.desc.sweep = (uint32_t)s.done;
        int rc = b->eng.upload_desc(k, s.desc);
        if (rc) return rc;
    }
    return ISING_OK;
}

int check_batch(ising_batch_t b, int32_t idx)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    if (idx < 0 || idx >= b->capacity || !b->slots[idx].used) return fail(ISING_EINVAL, "bad slot %d", idx);
    return ISING_OK;
}

int batch_sweeps_done(ising_batch_t b, int32_t idx, int64_t* done)
{
    uint32_t sw = 0;
    CK(cudaMemcpyAsync(&sw, &b->eng.d_desc[idx].sweep, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    int rc = b->eng.check_status();
    if (rc) return rc;
    *done = sw;
    return ISING_OK;
}
}  // namespace

int ising_batch_create_ex(ising_batch_t* out, int32_t capacity, int64_t max_L, int64_t arena_bytes, int32_t threads,
                          void* stream)
{
    if (!out) return fail(ISING_EINVAL, "null output");
    if (capacity < 1 || capacity > (1 << 20)) return fail(ISING_EINVAL, "capacity out of range");
    if (max_L < 64 || max_L % 64 || max_L > kPackedMaxL) return fail(ISING_EINVAL, "max_L must be a multiple of 64");
    if (threads == 0) threads = 256;
    if (threads != 128 && threads != 256 && threads != 512)
        return fail(ISING_EINVAL, "threads must be 128, 256 or 512");
    if (arena_bytes < 256) return fail(ISING_EINVAL, "arena too small");
    ising_batch_t b = new ising_batch_s();
    b->capacity = capacity;
    b->max_L = max_L;
    b->slots.resize((size_t)capacity);
    int rc = make_stream(stream, &b->stream, &b->own_stream);
    if (rc) {
        delete b;
        return rc;
    }
    // stage size: the largest tile any admissible lattice can use by default (whole
    // rows, or the built-in column blocks of rows too long for them); a column block
    // asked for in ising_batch_add_tiled must fit this too
    int64_t stage = 0;
    for (int64_t L = 64; L <= max_L; L += 64) {
        for (int tr = 2; tr <= kMaxTileRows; tr *= 2)
            if (tile_rows_ok(L, tr)) stage = std::max(stage, stage_bytes_for(L, tr));
        if (L % 256 == 0 && !whole_rows_ok(L)) stage = std::max(stage, stage_bytes_for(L, 2, default_tile_words(L)));
    }
    rc = b->eng.setup(capacity, (int)stage, threads, b->stream);
    if (!rc) rc = b->arena.init(arena_bytes);
    if (!rc) {
        cudaError_t e = cudaMalloc(&b->d_me, 2 * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_mom, 6 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_sums, 11 * sizeof(uint64_t));
        if (e != cudaSuccess) rc = cuda_fail(e, "batch buffers");
    }
    if (!rc) rc = rebuild_tiles(b);
    if (rc) {
        ising_batch_free(b);
        return rc;
    }
    *out = b;
    return ISING_OK;
}

int ising_batch_add(ising_batch_t b, int64_t L, double beta, uint64_t seed, int32_t start, int64_t sweeps,
                    int32_t tile_rows, int32_t* idx)
{
    return ising_batch_add_tiled(b, L, beta, seed, start, sweeps, tile_rows, 0, idx);
}

// Tile height for a lattice of a batch known in full at creation: the tallest whole-row
// tile of at most 8,192 words (256 rows at most, a power of two the stage holds), or 0
// (the built-in height) for sides that take column blocks.  Taller tiles give each warp
// more words per tile, so the per-tile costs (the stage handoff, the last partial drain
// of each warp's queue) weigh less; they pay once the batch holds enough of them for
// every CTA of the persistent grid (ising_batch_create).
static int tall_tile_rows(int64_t L)
{
    const int64_t W = L / 64;
    if (default_tile_words(L) != (int)W) return 0;
    int best = 0;
    for (int tr = 2; tr <= kMaxTileRows; tr *= 2)
        if (tile_rows_ok(L, tr) && (int64_t)tr * W <= 8192) best = tr;
    return best;
}

int ising_batch_create(ising_batch_t* out, int32_t count, const int64_t* L, const double* beta, const uint64_t* seed,
                       const int32_t* start)
{
    if (!out || !L || !beta || !seed || !start) return fail(ISING_EINVAL, "null argument");
    if (count < 1 || count > (1 << 20)) return fail(ISING_EINVAL, "count %d outside 1 .. 2^20", count);
    // every argument is checked before any device work
    int64_t max_L = 64, arena = 0;
    for (int32_t k = 0; k < count; ++k) {
        uint64_t T[2];
        if (L[k] < 64 || L[k] % 64 || !packed_L_ok(L[k]))
            return fail(ISING_EINVAL, "lattice %d: L = %lld is not a packed side", k, (long long)L[k]);
        if (!thresholds(beta[k], T)) return fail(ISING_EINVAL, "lattice %d: beta must be finite and >= 0", k);
        if (start[k] != ISING_HOT && start[k] != ISING_COLD) return fail(ISING_EINVAL, "lattice %d: bad start", k);
        max_L = std::max(max_L, L[k]);
        arena += FreeList::round_up((int64_t)sizeof(uint32_t) * 2 * L[k] * (L[k] / 64));
    }
    ising_batch_t b = nullptr;
    // CTA size as for single handles: one 512-thread CTA per SM once a side reaches 16,384
    int rc = ising_batch_create_ex(&b, count, max_L, arena, max_L >= 16384 ? 512 : 256, nullptr);
    if (rc) return rc;
    b->growable = true;
    // tall tiles when they still give every CTA of the persistent grid two tiles or more
    int64_t tall_tiles = 0;
    for (int32_t k = 0; k < count; ++k) {
        const int tr = tall_tile_rows(L[k]);
        tall_tiles += tr ? L[k] / tr : lattice_tiles(L[k], default_tile_rows(L[k], b->eng.threads), 0);
    }
    const bool tall = tall_tiles >= 2 * (int64_t)b->eng.grid;
    constexpr int64_t kFirstHistory = 1024;  // sweeps of history at admission, doubled as needed
    for (int32_t k = 0; k < count && !rc; ++k) {
        int32_t idx = -1;
        rc = ising_batch_add(b, L[k], beta[k], seed[k], start[k], kFirstHistory, tall ? tall_tile_rows(L[k]) : 0,
                             &idx);
    }
    if (rc) {
        const std::string msg = t_error;
        ising_batch_free(b);
        t_error = msg;
        return rc;
    }
    *out = b;
    return ISING_OK;
}

int ising_batch_add_tiled(ising_batch_t b, int64_t L, double beta, uint64_t seed, int32_t start, int64_t sweeps,
                          int32_t tile_rows, int32_t tile_words, int32_t* idx)
{
    if (!b || !idx) return fail(ISING_EINVAL, "null argument");
    uint64_t T[2];
    if (!thresholds(beta, T)) return fail(ISING_EINVAL, "beta must be finite and >= 0");
    if (L < 64 || L % 64 || L > b->max_L) return fail(ISING_EINVAL, "L must be a multiple of 64 and <= max_L");
    if (!packed_L_ok(L)) return fail(ISING_EINVAL, "no tile of L = %lld rows fits a shared-memory stage", (long long)L);
    if (start != ISING_HOT && start != ISING_COLD) return fail(ISING_EINVAL, "bad start");
    if (sweeps < 1 || sweeps > kMaxSweeps) return fail(ISING_EINVAL, "sweeps out of range");
    const int W = (int)(L / 64);
    if (tile_words == 0) tile_words = default_tile_words(L);
    if (tile_words == W) {
        if (tile_rows == 0 || !tile_rows_ok(L, tile_rows)) tile_rows = default_tile_rows(L, b->eng.threads);
    } else {
        if (tile_rows == 0) tile_rows = 2;
        if (!tile_ok(L, tile_rows, tile_words))
            return fail(ISING_EINVAL, "tile of %d rows x %d words is not a column block of L = %lld", tile_rows,
                        tile_words, (long long)L);
    }
    if (stage_bytes_for(L, tile_rows, tile_words) > b->eng.stage_bytes)
        return fail(ISING_EINVAL, "tile of %d rows x %d words exceeds the batch's stage", tile_rows, tile_words);
    int slot = -1;
    for (int k = 0; k < b->capacity; ++k)
        if (!b->slots[k].used) {
            slot = k;
            break;
        }
    if (slot < 0) return fail(ISING_EBUSY, "all %d slots in use", b->capacity);
    const int64_t plane_words = L * (L / 64);
    const int64_t plane_bytes = (int64_t)sizeof(uint32_t) * 2 * plane_words;
    // a growable batch keeps histories apart from the arena (they are resized); else the
    // history of `sweeps` sweeps follows the planes in the arena
    const int64_t bytes = plane_bytes + (b->growable ? 0 : 16 * sweeps);
    int64_t* own_hist = nullptr;
    if (b->growable) CK(cudaMalloc(&own_hist, 16 * (size_t)sweeps));
    const int64_t off = b->arena.alloc(bytes);
    if (off < 0) {
        cudaFree(own_hist);
        return fail(ISING_ENOMEM, "arena full: %lld of %lld bytes used, need %lld", (long long)b->arena.used,
                    (long long)b->arena.size, (long long)bytes);
    }
    auto& s = b->slots[slot];
    s.used = true;
    s.L = L;
    s.off = off;
    s.bytes = bytes;
    s.sweeps_cap = sweeps;
    s.own_hist = own_hist;
    s.done = 0;
    uint32_t* planes = reinterpret_cast<uint32_t*>(b->arena.base + off);
    LatticeDesc& d = s.desc;
    d = LatticeDesc{};
    d.plane[0] = planes;
    d.plane[1] = planes + plane_words;
    d.hist = own_hist ? own_hist : reinterpret_cast<int64_t*>(b->arena.base + off + plane_bytes);
    d.key = seed;
    d.L = (int32_t)L;
    d.W = (int32_t)(L / 64);
    set_thresholds(d, T);
    d.tile_rows = tile_rows;
    d.halo_rows = halo_rows_for(L / 64);
    d.tile_words = tile_words;
    d.sweep = 0;
    d.target = b->growable ? kNoTarget : (uint32_t)sweeps;
    if (tile_words != W) b->eng.allow_blocks();
    d.active = 1;
    cudaError_t e = launch_packed_init(d.plane[0], d.plane[1], L, seed, start, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    int rc = b->eng.upload_desc(slot, d);
    if (!rc) rc = rebuild_tiles(b);
    if (rc) return rc;
    *idx = slot;
    return ISING_OK;
}

int ising_batch_remove(ising_batch_t b, int32_t idx)
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    auto& s = b->slots[idx];
    s.desc.active = 0;
    rc = b->eng.upload_desc(idx, s.desc);
    if (rc) return rc;
    s.used = false;
    b->arena.release(s.off, s.bytes);
    if (s.own_hist) {
        CK(cudaStreamSynchronize(b->stream));  // the slot's pending sweeps may still write it
        cudaFree(s.own_hist);
        s.own_hist = nullptr;
    }
    return rebuild_tiles(b);
}

int ising_batch_run(ising_batch_t b, int64_t sweeps, int32_t graph_sweeps)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    if (sweeps < 0) return fail(ISING_EINVAL, "sweeps must be >= 0");
    if (graph_sweeps > 0 && sweeps % graph_sweeps)
        return fail(ISING_EINVAL, "sweeps %lld not a multiple of graph_sweeps %d", (long long)sweeps, graph_sweeps);
    if (b->growable) {
        for (const auto& s : b->slots)
            if (s.used && sweeps > kMaxSweeps - s.done)
                return fail(ISING_EINVAL, "sweep total beyond 2^32 - 2");
        int rc = grow_histories(b, sweeps);
        if (rc) return rc;
    }
    int rc = b->eng.run(sweeps, graph_sweeps);
    if (rc) return rc;
    if (b->growable)
        for (auto& s : b->slots)
            if (s.used) s.done += sweeps;
    return ISING_OK;
}

int ising_batch_sweeps_done(ising_batch_t b, int32_t idx, int64_t* sweeps_done)
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    if (!sweeps_done) return fail(ISING_EINVAL, "null output");
    return batch_sweeps_done(b, idx, sweeps_done);
}

int ising_batch_progress(ising_batch_t b, int64_t* sweeps_done, int32_t n)
{
    if (!b || !sweeps_done || n < 0 || n > b->capacity) return fail(ISING_EINVAL, "bad argument");
    std::vector<LatticeDesc> d((size_t)std::max(n, 1));
    if (n) CK(cudaMemcpyAsync(d.data(), b->eng.d_desc, sizeof(LatticeDesc) * (size_t)n, cudaMemcpyDeviceToHost,
                              b->stream));
    int rc = b->eng.check_status();
    if (rc) return rc;
    for (int32_t k = 0; k < n; ++k) sweeps_done[k] = b->slots[k].used ? (int64_t)d[k].sweep : -1;
    return ISING_OK;
}

int ising_batch_set_cluster(ising_batch_t b, int32_t mode)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    if (mode != ISING_CLUSTER_OFF && mode != ISING_CLUSTER_AUTO && mode != ISING_CLUSTER_ALWAYS)
        return fail(ISING_EINVAL, "cluster mode %d is not 0, 1 or 2", mode);
    b->cluster_mode = mode;
    return update_cluster(b);
}

int ising_batch_cluster_size(ising_batch_t b, int32_t* cluster_size)
{
    if (!b || !cluster_size) return fail(ISING_EINVAL, "null argument");
    *cluster_size = b->eng.cluster.C;
    return ISING_OK;
}

int ising_batch_specialized(ising_batch_t b, int32_t* specialized)
{
    if (!b || !specialized) return fail(ISING_EINVAL, "null argument");
    *specialized = b->eng.fixed_multi ? 1 : 0;
    return ISING_OK;
}

int ising_batch_gather(ising_batch_t b, int32_t n, const int32_t* idx, int64_t* out)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    if (n < 0 || n > b->capacity) return fail(ISING_EINVAL, "n %d outside 0 .. capacity %d", n, b->capacity);
    if (n == 0) return ISING_OK;
    if (!idx || !out) return fail(ISING_EINVAL, "null argument");
    for (int32_t k = 0; k < n; ++k)
        if (idx[k] < 0 || idx[k] >= b->capacity || !b->slots[idx[k]].used)
            return fail(ISING_EINVAL, "bad slot %d", idx[k]);
    CK(launch_gather(b->eng.d_desc, idx, n, out, b->stream));
    return ISING_OK;
}

int ising_batch_observables_ex(ising_batch_t b, int32_t idx, int64_t* M, int64_t* E, int64_t* sweeps_done)
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    int64_t done = 0;
    rc = batch_sweeps_done(b, idx, &done);
    if (rc) return rc;
    const auto& d = b->slots[idx].desc;
    int64_t me[2];
    if (done == 0) {
        CK(launch_packed_observe(d.plane[0], d.plane[1], d.L, b->d_me, b->stream));
        CK(cudaMemcpyAsync(me, b->d_me, sizeof(me), cudaMemcpyDeviceToHost, b->stream));
    } else {
        CK(cudaMemcpyAsync(me, d.hist + 2 * (done - 1), sizeof(me), cudaMemcpyDeviceToHost, b->stream));
    }
    CK(cudaStreamSynchronize(b->stream));
    if (M) *M = me[0];
    if (E) *E = me[1];
    if (sweeps_done) *sweeps_done = done;
    return ISING_OK;
}

int ising_batch_observables(ising_batch_t b, int32_t idx, int64_t* M, int64_t* E)
{
    return ising_batch_observables_ex(b, idx, M, E, nullptr);
}

int ising_batch_history(ising_batch_t b, int32_t idx, int64_t first, int64_t count, int64_t* M, int64_t* E)
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    int64_t done = 0;
    rc = batch_sweeps_done(b, idx, &done);
    if (rc) return rc;
    if (first < 0 || count < 0 || first > done || count > done - first)
        return fail(ISING_EINVAL, "history range beyond sweeps done");
    std::vector<int64_t> buf(2 * (size_t)count);
    const auto& d = b->slots[idx].desc;
    if (count) CK(cudaMemcpyAsync(buf.data(), d.hist + 2 * first, sizeof(int64_t) * buf.size(),
                                  cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int64_t k = 0; k < count; ++k) {
        if (M) M[k] = buf[2 * k];
        if (E) E[k] = buf[2 * k + 1];
    }
    return ISING_OK;
}

int ising_batch_moments(ising_batch_t b, int32_t idx, int64_t burn_in, double out[6], uint64_t sums[11])
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    if (!out) return fail(ISING_EINVAL, "null output");
    int64_t done = 0;
    rc = batch_sweeps_done(b, idx, &done);
    if (rc) return rc;
    if (burn_in < 0 || burn_in >= done) return fail(ISING_EINVAL, "no samples after burn-in");
    const auto& d = b->slots[idx].desc;
    CK(launch_moments(d.hist, burn_in, done - burn_in, (int64_t)d.L * d.L, b->d_mom, b->d_sums, b->stream));
    double m[6];
    uint64_t s[11];
    CK(cudaMemcpyAsync(m, b->d_mom, sizeof(m), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(s, b->d_sums, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    memcpy(out, m, sizeof(m));
    if (sums) memcpy(sums, s, sizeof(s));
    return ISING_OK;
}

int ising_batch_get_lattice(ising_batch_t b, int32_t idx, int8_t* out)
{
    int rc = check_batch(b, idx);
    if (rc) return rc;
    if (!out) return fail(ISING_EINVAL, "null output");
    rc = b->eng.check_status();
    if (rc) return rc;
    const auto& d = b->slots[idx].desc;
    return packed_to_host(d.plane[0], d.plane[1], d.L, out, b->stream);
}

int ising_batch_usage(ising_batch_t b, int64_t* arena_used, int32_t* slots_used)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    if (arena_used) *arena_used = b->arena.used;
    if (slots_used) {
        int32_t n = 0;
        for (const auto& s : b->slots) n += s.used ? 1 : 0;
        *slots_used = n;
    }
    return ISING_OK;
}

int ising_batch_synchronize(ising_batch_t b)
{
    if (!b) return fail(ISING_EINVAL, "null batch");
    return b->eng.check_status();
}

int ising_batch_free(ising_batch_t b)
{
    if (!b) return ISING_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->eng.destroy();
    b->arena.destroy();
    for (auto& s : b->slots) cudaFree(s.own_hist);
    cudaFree(b->d_me);
    cudaFree(b->d_mom);
    cudaFree(b->d_sums);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return ISING_OK;
}

// ==================================================================== autotune
int ising_autotune(int64_t L, int32_t* tile_rows, int32_t* threads, double* ms)
{
    if (!tile_rows || !threads) return fail(ISING_EINVAL, "null output");
    if (!packed_L_ok(L)) return fail(ISING_EINVAL, "L must be a multiple of 64 that a tile can hold");
    if (!whole_rows_ok(L)) return fail(ISING_EINVAL, "the autotuner times whole-row tiles (L <= 272896)");
    // time as many copies of the lattice as it takes to give every SM work (up to
    // 2^26 sites or 64 copies), as in a batch where this size is common
    int copies = 1;
    while (copies < 64 && (int64_t)copies * L * L < (1ll << 26)) copies *= 2;
    // sweeps per timing: about 2^32 site updates (at least 16, at most 256), so that a
    // candidate's time is long against launch jitter; each candidate is timed twice and
    // its better time kept
    const int64_t per_sweep_sites = (int64_t)copies * L * L;
    const int reps = (int)std::min<int64_t>(256, std::max<int64_t>(16, (1ll << 32) / per_sweep_sites));
    double best = 1e300;
    int best_tr = 0, best_th = 0;
    const int thread_opts[2] = {256, 512};
    for (int ti = 0; ti < 2; ++ti) {
        ising_batch_t b = nullptr;
        const int64_t per = (int64_t)sizeof(uint32_t) * 2 * L * (L / 64) + 16 * (2 * reps + 4) + 512;
        int rc = ising_batch_create_ex(&b, copies, L, per * copies + 4096, thread_opts[ti], nullptr);
        if (rc) return rc;
        b->cluster_mode = ISING_CLUSTER_OFF;  // the tiled kernel's shapes are what is timed
        for (int tr = 2; tr <= kMaxTileRows; tr *= 2) {
            if (!tile_rows_ok(L, tr)) continue;  // whole rows only
            std::vector<int32_t> idx((size_t)copies, -1);
            for (int k = 0; k < copies && !rc; ++k)
                rc = ising_batch_add(b, L, 0.4406868, 12345 + k, ISING_HOT, 2 * reps + 4, tr, &idx[(size_t)k]);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            if (!rc) rc = b->eng.run(2, 0);  // warm-up
            float t = 1e30f;
            for (int m = 0; m < 2 && !rc; ++m) {
                cudaEventRecord(e0, b->stream);
                rc = b->eng.run(reps, 0);
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float tm = 0;
                cudaEventElapsedTime(&tm, e0, e1);
                t = std::min(t, tm);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (!rc) rc = b->eng.check_status();
            if (rc) {
                ising_batch_free(b);
                return rc;
            }
            const double per_sweep = (double)t / reps;
            if (per_sweep < best) {
                best = per_sweep;
                best_tr = tr;
                best_th = thread_opts[ti];
            }
            for (int k = 0; k < copies; ++k) ising_batch_remove(b, idx[(size_t)k]);
        }
        ising_batch_free(b);
    }
    *tile_rows = best_tr;
    *threads = best_th;
    if (ms) *ms = best / copies;
    return ISING_OK;
}

// ================================================================ self-test
int ising_selftest_timeout(int64_t wait_cycles, int* observed)
{
    if (!observed || wait_cycles < 1000 || wait_cycles > 4000000000ll) return fail(ISING_EINVAL, "bad argument");
    ising_t h = nullptr;
    int rc = ising_init_ex(&h, 256, 0.44, 1, ISING_HOT, ISING_PACKED, nullptr);
    if (rc) return rc;
    // every tile barrier of this launch expects 16 bytes that are never sent
    cudaError_t e = launch_packed_half_sweep(h->eng.table(), 0, 0, h->eng.d_status, h->eng.grid, h->eng.threads,
                                             h->eng.stage_bytes, h->stream, (long long)wait_cycles, 16u);
    if (e != cudaSuccess) {
        ising_free(h);
        return cuda_fail(e, "self-test launch");
    }
    *observed = h->eng.check_status();
    // the context must still be usable: a normal sweep now completes cleanly
    rc = ising_sweep(h, 1);
    if (!rc) rc = ising_synchronize(h);
    ising_free(h);
    return rc;
}

// ============================================================ device blocks
int ising_dev_philox(uint64_t key, const uint32_t ctr[4], int64_t nblocks, uint32_t* out, void* stream)
{
    if (!ctr || !out || nblocks < 0) return fail(ISING_EINVAL, "bad argument");
    CK(launch_philox_words(key, ctr, nblocks, out, (cudaStream_t)stream));
    return ISING_OK;
}

}  // extern "C"

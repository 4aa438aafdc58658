// Sweeps of caller-owned packed lattices that allocate no device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// graph is being captured (allocation is not a capturable operation), plugins
// that live inside another runtime's fixed memory pool, and real-time loops
// whose memory must be fixed after start-up.  This entry point lets them run
// the packed checkerboard sweep on memory they already own: they pass the bit
// planes and an M/E output array; the small scratch the sweep kernel needs
// (lattice descriptors, tile table, lattice count, status word) lives in one
// file-scope __device__ array, sized for at most kNoAllocMaxLattices lattices.
// Every GPU that loads this library holds that array until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (and sets the sweep kernel's shared-memory limit); make
// that first call before any stream capture.  All calls share the array and it
// keeps the last call's contents: each call rewrites the descriptors and
// clears the status word before its sweeps, and calls whose work overlaps on
// the GPU (different streams, no ordering between them) race on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ising.h"
#include "ising_internal.cuh"

namespace ising {
namespace {

constexpr int kNoAllocMaxLattices = 64;
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxDevices = 64;
constexpr int64_t kNoAllocStageCap = kStageCapBytes;  // the handle API's per-stage limit

struct NoAllocScratch {
    LatticeDesc desc[kNoAllocMaxLattices];
    int32_t tile_start[kNoAllocMaxLattices + 1];
    int32_t count;
    int32_t status;
};
// The size the header states (64 descriptors of 80 bytes, the tile table, count and
// status: 5,388 bytes, padded to 5,392).
static_assert(sizeof(LatticeDesc) == 80, "descriptor size behind the stated scratch size");
static_assert(sizeof(NoAllocScratch) == 5392, "scratch size stated in the header");

// The scratch of every call.  In host code `g_noalloc_scratch` names a host-side
// shadow, not device memory; host code must use the address that
// cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

struct SetupParams {
    LatticeDesc desc[kNoAllocMaxLattices];
    int32_t tile_start[kNoAllocMaxLattices + 1];
    int32_t count;
};

// Writes this call's descriptors into the scratch and clears the status word.
__global__ void noalloc_setup_kernel(NoAllocScratch* s, const SetupParams p)
{
    const int t = threadIdx.x;
    if (t < p.count) s->desc[t] = p.desc[t];
    if (t <= p.count) s->tile_start[t] = p.tile_start[t];
    if (t == 0) {
        s->count = p.count;
        s->status = kStatusOk;
    }
}

struct DeviceState {
    NoAllocScratch* scratch = nullptr;
    int sms = 0;
};

std::mutex g_mu;
DeviceState g_dev[kNoAllocMaxDevices];

int set_error(int code, const char* msg)
{
    set_last_error(msg);
    return code;
}

int64_t halo_rows(int64_t W) { return (W % 4 == 0) ? 1 : 4; }

int64_t stage_bytes(int64_t L, int tr)
{
    const int64_t W = L / 64;
    return (stage_words((int32_t)W, tr, (int32_t)halo_rows(W)) * 4 + 15) / 16 * 16;
}

int tile_rows_for(int64_t L)
{
    const int64_t W = L / 64;
    int tr = 64;
    while (tr > 4 && (int64_t)tr * W > 4096) tr >>= 1;
    while (tr > 4 && (L % tr != 0 || stage_bytes(L, tr) > kNoAllocStageCap)) tr >>= 1;
    return tr;
}

// Once per device, with that device current: the scratch's device address, the
// kernel's shared-memory limit (the largest stage any call can use) and the SM count.
int device_setup(int dev, DeviceState** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState& st = g_dev[dev];
    if (!st.scratch) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
        const int stage = (int)kNoAllocStageCap;
        const size_t smem = (size_t)packed_smem_header_bytes(kNoAllocThreads) + 2 * (size_t)stage;
        e = packed_set_smem_limit(kNoAllocThreads, smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = packed_occupancy(kNoAllocThreads, smem, &per_sm);
        if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
        if (per_sm < 1) return set_error(ISING_ECUDA, "sweep kernel does not fit on this device");
        e = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
        st.scratch = static_cast<NoAllocScratch*>(ptr);
    }
    *out = &st;
    return ISING_OK;
}

}  // namespace
}  // namespace ising

extern "C" int ising_sweep_packed_noalloc(int32_t count, uint32_t* const* black, uint32_t* const* white,
                                          const int64_t* L, const double* beta, const uint64_t* seed,
                                          int64_t first_sweep, int64_t nsweeps, int64_t* const* me, void* stream,
                                          int32_t wait)
{
    using namespace ising;
    if (count < 1 || count > kNoAllocMaxLattices) {
        char buf[128];
        snprintf(buf, sizeof(buf), "count %d outside 1..%d lattices per call", count, kNoAllocMaxLattices);
        return set_error(ISING_EINVAL, buf);
    }
    if (!black || !white || !L || !beta || !seed || !me) return set_error(ISING_EINVAL, "null argument");
    if (first_sweep < 0 || nsweeps < 0 || first_sweep > 0xFFFFFFFEll || nsweeps > 0xFFFFFFFEll - first_sweep)
        return set_error(ISING_EINVAL, "sweep range outside 0 .. 2^32 - 2");
    SetupParams p;
    memset(&p, 0, sizeof(p));
    p.count = count;
    p.tile_start[0] = 0;
    int64_t tiles = 0, stage = 16;
    for (int k = 0; k < count; ++k) {
        if (L[k] < 64 || L[k] % 64 || L[k] > (1 << 20)) return set_error(ISING_EINVAL, "L must be a multiple of 64 in 64 .. 2^20");
        if (!black[k] || !white[k] || !me[k]) return set_error(ISING_EINVAL, "null plane or output pointer");
        uint64_t T[2];
        if (ising_thresholds(beta[k], T) != ISING_OK) return set_error(ISING_EINVAL, "beta must be finite and >= 0");
        const int tr = tile_rows_for(L[k]);
        if (stage_bytes(L[k], tr) > kNoAllocStageCap)
            return set_error(ISING_EINVAL, "L too large for a shared-memory tile: L <= 163840 (L % 256 == 0) or L <= 102336");
        LatticeDesc& d = p.desc[k];
        d.plane[0] = black[k];
        d.plane[1] = white[k];
        // the kernel writes sweep s at hist[2 s]; shift so that first_sweep lands on me[k][0]
        d.hist = me[k] - 2 * first_sweep;
        d.key = seed[k];
        d.L = (int32_t)L[k];
        d.W = (int32_t)(L[k] / 64);
        d.t2 = T[0] >= 4294967296ull ? 0xFFFFFFFFu : (uint32_t)T[0];
        d.t4 = T[1] >= 4294967296ull ? 0xFFFFFFFFu : (uint32_t)T[1];
        d.all2 = T[0] >= 4294967296ull ? 0xFFFFFFFFu : 0u;
        d.all4 = T[1] >= 4294967296ull ? 0xFFFFFFFFu : 0u;
        d.tile_rows = tr;
        d.halo_rows = (int32_t)halo_rows(L[k] / 64);
        d.tile_words = (int32_t)(L[k] / 64);  // whole rows
        d.sweep = (uint32_t)first_sweep;
        d.target = 0xFFFFFFFFu;
        d.active = 1;
        tiles += L[k] / tr;
        stage = stage_bytes(L[k], tr) > stage ? stage_bytes(L[k], tr) : stage;
        if (tiles > 0x7FFFFFFF) return set_error(ISING_EINVAL, "too many tiles");
        p.tile_start[k + 1] = (int32_t)tiles;
    }
    if (wait) {
        // a stream that is being captured cannot be synchronised; refuse before any work
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
        if (ce != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(ce));
        if (cs != cudaStreamCaptureStatusNone) return set_error(ISING_EINVAL, "wait != 0 on a stream that is being captured");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(ISING_EINVAL, "device index too large");
    DeviceState* st = nullptr;
    int rc = device_setup(dev, &st);
    if (rc) return rc;
    // persistent grid: as many CTAs as fit with this call's stage size
    const size_t smem = (size_t)packed_smem_header_bytes(kNoAllocThreads) + 2 * (size_t)stage;
    int per_sm = 0;
    e = packed_occupancy(kNoAllocThreads, smem, &per_sm);
    if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
    if (per_sm < 1) per_sm = 1;
    const int grid = per_sm * st->sms;
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_setup_kernel<<<1, kNoAllocMaxLattices + 1, 0, s>>>(st->scratch, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
    TileTable tt;
    tt.desc = st->scratch->desc;
    tt.tile_start = st->scratch->tile_start;
    tt.count = &st->scratch->count;
    int* status = &st->scratch->status;
    for (int64_t k = 0; k < nsweeps; ++k) {
        for (int c = 0; c < 2; ++c) {
            e = launch_packed_half_sweep(tt, c, (int)k, status, grid, kNoAllocThreads, (int)stage, s);
            if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
        }
    }
    if (wait) {
        int host_status = 0;
        e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(ISING_ECUDA, cudaGetErrorString(e));
        if (host_status == kStatusTimeout) return set_error(ISING_ETIMEOUT, "sweep kernel's bounded wait expired");
        if (host_status != kStatusOk) {
            char buf[96];
            snprintf(buf, sizeof(buf), "sweep kernel reported status %d (a bad tile or descriptor)", host_status);
            return set_error(ISING_ECUDA, buf);
        }
    }
    return ISING_OK;
}

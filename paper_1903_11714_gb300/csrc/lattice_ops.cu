// Start states, observables and layout conversions for the packed planes.
//
// Start states (the paper leaves them open; Sec. 4 simulates from random
// lattices): hot = each spin +1 iff its Philox word, drawn with the reserved
// sweep slot 0xFFFFFFFF and its own colour, is below 2^31; cold = all +1.
// Observables (Sec. 3 Hamiltonian with mu = 0, J = 1; Sec. 4.1 magnetisation):
// M = sum sigma = 2 * (#up) - N and E = -sum_bonds sigma sigma = 2 * (#anti-aligned
// bonds) - 2N, every bond counted from its white end.
#include "ising_internal.cuh"
#include "philox.cuh"

namespace ising {
namespace {


__global__ void packed_init_kernel(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start)
{
    const int64_t W = L / 64;
    const int64_t words = L * W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 2 * words;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int c = g >= words ? 1 : 0;
        const int64_t idx = g - c * words;
        uint32_t* plane = c ? white : black;
        if (start == 1) {
            plane[idx] = 0xFFFFFFFFu;
            continue;
        }
        // plane word idx = i * W + w holds plane indices 32 idx .. 32 idx + 31
        plane[idx] = hot_start_word((uint64_t)idx, (uint32_t)c, key);
    }
}

__global__ void set_pair_kernel(int64_t* p, int64_t a, int64_t b)
{
    p[0] = a;
    p[1] = b;
}

// Descriptor and tile-table updates carried as kernel parameters: the parameters are
// captured when the launch is enqueued, so the host's copy may change at once and
// nothing waits for the stream's earlier work.
__global__ void set_desc_kernel(LatticeDesc* dst, const LatticeDesc d)
{
    if (threadIdx.x == 0) *dst = d;
}

__global__ void set_tiles_kernel(int32_t* tile_start, int32_t* count_dst, const TileChunk c)
{
    for (int k = threadIdx.x; k < c.n; k += blockDim.x) tile_start[c.first + k] = c.v[k];
    if (threadIdx.x == 0 && c.count >= 0) *count_dst = c.count;
}

// (sweeps done, M, E) of batch slots a.idx[0 .. a.n): M and E of the lattice's last
// sweep, (0, 0) before any.
__global__ void gather_kernel(const LatticeDesc* desc, const GatherChunk a, int64_t* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const LatticeDesc& d = desc[a.idx[k]];
    const int64_t s = d.sweep;
    out[3 * k] = s;
    out[3 * k + 1] = s ? d.hist[2 * (s - 1)] : 0;
    out[3 * k + 2] = s ? d.hist[2 * (s - 1) + 1] : 0;
}

// Adds 2 * (#up) and 2 * (#anti-aligned bonds) into ME (pre-set to -N, -2N).
__global__ void packed_observe_kernel(const uint32_t* black, const uint32_t* white, int64_t L,
                                      unsigned long long* ME)
{
    const int64_t W = L / 64;
    const int64_t words = L * W;
    uint32_t ups = 0, anti = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / W, w = idx - i * W;
        const int64_t iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
        const uint32_t wh = white[idx];
        const uint32_t up = black[iu * W + w], down = black[id * W + w], same = black[idx];
        uint32_t hz;
        if ((i + 1) & 1) {
            const uint32_t nxt = black[i * W + (w + 1 == W ? 0 : w + 1)];
            hz = __funnelshift_r(same, nxt, 1);
        } else {
            const uint32_t prv = black[i * W + (w == 0 ? W - 1 : w - 1)];
            hz = __funnelshift_l(prv, same, 1);
        }
        ups += __popc(wh) + __popc(same);
        anti += __popc(wh ^ up) + __popc(wh ^ down) + __popc(wh ^ same) + __popc(wh ^ hz);
        if (ups > 0x40000000u || anti > 0x40000000u) {
            atomicAdd(&ME[0], 2ull * ups);
            atomicAdd(&ME[1], 2ull * anti);
            ups = anti = 0;
        }
    }
    const uint32_t u = __reduce_add_sync(0xffffffffu, ups);
    const uint32_t a = __reduce_add_sync(0xffffffffu, anti);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ME[0], 2ull * u);
        atomicAdd(&ME[1], 2ull * a);
    }
}

// int8 row-major (+1/-1) rows [row0, row0+nrows) -> planes.  `lat` points at row0.
__global__ void pack_kernel(const int8_t* lat, uint32_t* black, uint32_t* white, int64_t L, int64_t row0,
                            int64_t nrows)
{
    const int64_t W = L / 64;
    const int64_t words = nrows * W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 2 * words;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int c = g >= words ? 1 : 0;
        const int64_t idx = g - c * words;
        const int64_t il = idx / W, w = idx - il * W;
        const int64_t i = row0 + il;
        const int r = (int)((i + c) & 1);
        const int8_t* row = lat + il * L;
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) bits |= (row[2 * (32 * w + b) + r] > 0 ? 1u : 0u) << b;
        (c ? white : black)[i * W + w] = bits;
    }
}

// planes rows [row0, row0+nrows) -> int8 row-major at `lat` (row0 first).
__global__ void unpack_kernel(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                              int64_t nrows)
{
    const int64_t W = L / 64;
    const int64_t words = nrows * W;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t il = idx / W, w = idx - il * W;
        const int64_t i = row0 + il;
        int8_t* row = lat + il * L + 64 * w;
        const uint32_t bw[2] = {black[i * W + w], white[i * W + w]};
        for (int c = 0; c < 2; ++c) {
            const int r = (int)((i + c) & 1);
            for (int b = 0; b < 32; ++b) row[2 * b + r] = ((bw[c] >> b) & 1u) ? (int8_t)1 : (int8_t)-1;
        }
    }
}

__global__ void philox_words_kernel(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                                    uint32_t* out)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t q = ((uint64_t)c1 << 32 | c0) + (uint64_t)b;
        uint32_t x[4];
        philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), c2, c3, key, x);
        for (int m = 0; m < 4; ++m) out[4 * b + m] = x[m];
    }
}

int grid_for(int64_t work, int threads)
{
    const int64_t want = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_set_desc(LatticeDesc* dst, const LatticeDesc& d, cudaStream_t s)
{
    set_desc_kernel<<<1, 32, 0, s>>>(dst, d);
    return cudaGetLastError();
}

cudaError_t launch_set_tiles(int32_t* tile_start, int32_t* count_dst, const int32_t* v, int32_t n, int32_t count,
                             cudaStream_t s)
{
    int32_t first = 0;
    do {
        TileChunk c;
        c.first = first;
        c.n = n - first < TileChunk::kMax ? n - first : TileChunk::kMax;
        c.count = first + c.n >= n ? count : -1;  // the count goes with the last chunk
        for (int k = 0; k < c.n; ++k) c.v[k] = v[first + k];
        set_tiles_kernel<<<1, 256, 0, s>>>(tile_start, count_dst, c);
        first += c.n;
    } while (first < n);
    return cudaGetLastError();
}

cudaError_t launch_gather(const LatticeDesc* desc, const int32_t* idx, int32_t n, int64_t* out, cudaStream_t s)
{
    for (int32_t first = 0; first < n; first += GatherChunk::kMax) {
        GatherChunk a;
        a.n = n - first < GatherChunk::kMax ? n - first : GatherChunk::kMax;
        for (int k = 0; k < a.n; ++k) a.idx[k] = idx[first + k];
        gather_kernel<<<(a.n + 127) / 128, 128, 0, s>>>(desc, a, out + 3 * (int64_t)first);
    }
    return cudaGetLastError();
}

cudaError_t launch_packed_init(uint32_t* black, uint32_t* white, int64_t L, uint64_t key, int start, cudaStream_t s)
{
    packed_init_kernel<<<grid_for(2 * L * (L / 64), 256), 256, 0, s>>>(black, white, L, key, start);
    return cudaGetLastError();
}

cudaError_t launch_packed_observe(const uint32_t* black, const uint32_t* white, int64_t L, int64_t* ME,
                                  cudaStream_t s)
{
    set_pair_kernel<<<1, 1, 0, s>>>(ME, -L * L, -2 * L * L);
    packed_observe_kernel<<<grid_for(L * (L / 64), 256), 256, 0, s>>>(black, white, L,
                                                                     reinterpret_cast<unsigned long long*>(ME));
    return cudaGetLastError();
}

cudaError_t launch_pack(const int8_t* lat, uint32_t* black, uint32_t* white, int64_t L, int64_t row0,
                        int64_t nrows, cudaStream_t s)
{
    pack_kernel<<<grid_for(2 * nrows * (L / 64), 256), 256, 0, s>>>(lat, black, white, L, row0, nrows);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t* black, const uint32_t* white, int8_t* lat, int64_t L, int64_t row0,
                          int64_t nrows, cudaStream_t s)
{
    unpack_kernel<<<grid_for(nrows * (L / 64), 256), 256, 0, s>>>(black, white, lat, L, row0, nrows);
    return cudaGetLastError();
}

cudaError_t launch_philox_words(uint64_t key, const uint32_t* ctr4, int64_t n, uint32_t* out, cudaStream_t s)
{
    philox_words_kernel<<<grid_for(n, 256), 256, 0, s>>>(key, ctr4[0], ctr4[1], ctr4[2], ctr4[3], n, out);
    return cudaGetLastError();
}

}  // namespace ising

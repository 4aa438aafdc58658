// Plain int8 checkerboard half-sweep: the GPU analogue of the paper's
// UpdateNaive (Algorithm 1) on a row-major L x L lattice of +1/-1 bytes, with
// the same Philox keying, integer thresholds and fused M/E counts as the
// bit-packed kernel, so both reach the same chain bit for bit.
//
// The start-state kernel works on 8-byte chunks (columns 8g .. 8g+7): the four
// sites of each colour in a chunk lie in one plane word and take their start spins
// from its first random word.  The half-sweep works on 64-byte row segments (the
// 32 target sites of one plane word) when L % 64 == 0, else on 8-byte chunks; both
// run the bit-sliced test of word_update.cuh on per-site class masks.
#include "ising_internal.cuh"
#include "word_update.cuh"

namespace ising {
namespace {


__device__ __forceinline__ int sbyte(uint64_t v, int k)
{
    return (int)(int8_t)(uint8_t)(v >> (8 * k));
}

__global__ void int8_init_kernel(int8_t* lat, int64_t L, uint64_t key, int start)
{
    const int64_t G = L / 8;
    const int64_t chunks = L * G;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < chunks;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / G, g = idx - i * G;
        uint64_t v = 0;
        if (start == 1) {
            v = 0x0101010101010101ull;
        } else {
            // the chunk's 4 sites of each colour have plane indices p0 .. p0+3, all in
            // plane word p0 >> 5 (p0 is a multiple of 4)
            const uint64_t p0 = (uint64_t)i * (uint64_t)(L / 2) + 4ull * (uint64_t)g;
            for (int c = 0; c < 2; ++c) {
                const uint32_t up_bits = hot_start_word(p0 >> 5, (uint32_t)c, key) >> (p0 & 31);
                const int r = (int)((i + c) & 1);
                for (int b = 0; b < 4; ++b) {
                    const uint64_t byte = ((up_bits >> b) & 1u) ? 0x01ull : 0xFFull;
                    v |= byte << (8 * (2 * b + r));
                }
            }
        }
        *reinterpret_cast<uint64_t*>(lat + i * L + 8 * g) = v;
    }
}

__device__ __forceinline__ int sbyte32(uint32_t v, int k)
{
    return (int)(int8_t)(uint8_t)(v >> (8 * k));
}

__device__ __forceinline__ void block_add_pair(long long a, long long b, int64_t* slot)
{
    __shared__ long long red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sa = 0, sb = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sa += red[0][k];
            sb += red[1][k];
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)sa);
        atomicAdd(reinterpret_cast<unsigned long long*>(slot + 1), (unsigned long long)sb);
    }
}

__global__ void int8_half_sweep_seg64_kernel(int8_t* lat, int64_t L, uint64_t key, uint32_t t2, uint32_t t4, uint32_t all2,
                                       uint32_t all4, uint32_t sweep, int colour, int64_t* hist_slot)
{
    // One thread owns a 64-byte segment of a row: columns 64g .. 64g+63, i.e. the
    // 32 target sites j = 64g + 2b + r (b = 0..31) whose plane indices p = i*L/2 +
    // 32g + b form plane word i*L/64 + g, drawn from the calls q = i*L/8 + 8g + 0..7.
    const int64_t G = L / 64;
    const int64_t segs = L * G;
    if (colour == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        hist_slot[0] = 0;  // opened here, filled by the colour-1 pass of the same sweep
        hist_slot[1] = 0;
    }
    const PhiloxWordConsts pc = philox_consts(key, 0u, sweep, (uint32_t)colour);
    const uint32_t thr[2] = {t2, t4};
    const uint32_t zero2 = (t2 == 0u && all2 == 0u) ? ~0u : 0u, zero4 = (t4 == 0u && all4 == 0u) ? ~0u : 0u;
    long long m_acc = 0, e_acc = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < segs;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / G, g = idx - i * G;
        const int64_t iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
        const int r = (int)((i + colour) & 1);
        int8_t* row = lat + i * L + 64 * g;
        uint32_t cw[16], uw[16], dw[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 c4 = reinterpret_cast<const uint4*>(row)[k];
            const uint4 u4 = reinterpret_cast<const uint4*>(lat + iu * L + 64 * g)[k];
            const uint4 d4 = reinterpret_cast<const uint4*>(lat + id * L + 64 * g)[k];
            cw[4 * k] = c4.x; cw[4 * k + 1] = c4.y; cw[4 * k + 2] = c4.z; cw[4 * k + 3] = c4.w;
            uw[4 * k] = u4.x; uw[4 * k + 1] = u4.y; uw[4 * k + 2] = u4.z; uw[4 * k + 3] = u4.w;
            dw[4 * k] = d4.x; dw[4 * k + 1] = d4.y; dw[4 * k + 2] = d4.z; dw[4 * k + 3] = d4.w;
        }
        // the one neighbour outside the segment: column 64g-1 (r = 0) or 64g+64 (r = 1)
        const int64_t edge_col = r ? (g + 1 == G ? 0 : 64 * g + 64) : (g == 0 ? L - 1 : 64 * g - 1);
        const int edge = lat[i * L + edge_col];
        const uint64_t q0 = (uint64_t)i * (uint64_t)(L / 8) + 8ull * (uint64_t)g;
        const PhiloxWordConsts pcw =
            L <= 131072 ? pc : philox_consts(key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
        // per-site classes of the 32 target sites (bit b = site j = 64g + 2b + r):
        // h <= 0 always flips, h = 2 tests U < T2, h = 4 tests U < T4
        uint32_t alw = 0, h2m = 0, h4m = 0;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            if (rr != r) continue;
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                const int k = 2 * b + rr;
                const int s = sbyte32(cw[k >> 2], k & 3);
                const int left = k == 0 ? edge : sbyte32(cw[(k - 1) >> 2], (k - 1) & 3);
                const int right = k == 63 ? edge : sbyte32(cw[(k + 1) >> 2], (k + 1) & 3);
                const int h = s * (sbyte32(uw[k >> 2], k & 3) + sbyte32(dw[k >> 2], k & 3) + left + right);
                alw |= (h <= 0 ? 1u : 0u) << b;
                h2m |= (h == 2 ? 1u : 0u) << b;
                h4m |= (h == 4 ? 1u : 0u) << b;
            }
        }
        // the segment's target sites are plane word i * L/64 + g: q_lo = q0
        uint32_t lt[1] = {(h2m & all2) | (h4m & all4)};
        uint32_t und[1] = {(h2m & ~(all2 | zero2)) | (h4m & ~(all4 | zero4))};
        {
            // calls 0-1 (planes 0-7) as straight-line code: a 32-site word with most of its
            // sites tested needs both nearly always; the rest stop once the word is decided
            const uint32_t sel[1] = {h2m}, ql[1] = {(uint32_t)q0};
            bitsliced_below<1, 2, 0, 2, false, false>(und, lt, sel, sel, ql, pcw, key, thr);
            bitsliced_below<1, 2, 2, 8>(und, lt, sel, sel, ql, pcw, key, thr);
        }
        const uint32_t accm = alw | lt[0];
        uint32_t nw[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) nw[k] = cw[k];
        long long e_here = 0;
        // both parities are unrolled; r picks the target bytes (k = 2b + r)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            if (rr != r) continue;
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                const int k = 2 * b + rr;
                const int s = sbyte32(cw[k >> 2], k & 3);
                const int left = k == 0 ? edge : sbyte32(cw[(k - 1) >> 2], (k - 1) & 3);
                const int right = k == 63 ? edge : sbyte32(cw[(k + 1) >> 2], (k + 1) & 3);
                const int nn = sbyte32(uw[k >> 2], k & 3) + sbyte32(dw[k >> 2], k & 3) + left + right;
                const bool acc = (accm >> b) & 1u;
                if (acc) nw[k >> 2] ^= 0xFEu << (8 * (k & 3));  // 0x01 <-> 0xFF
                e_here -= (long long)(acc ? -s : s) * nn;
            }
        }
        bool changed = false;
#pragma unroll
        for (int k = 0; k < 16; ++k) changed |= nw[k] != cw[k];
        if (changed) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                reinterpret_cast<uint4*>(row)[k] = make_uint4(nw[4 * k], nw[4 * k + 1], nw[4 * k + 2], nw[4 * k + 3]);
        }
        if (colour == 1) {
            long long msum = 0;
#pragma unroll
            for (int k = 0; k < 64; ++k) msum += sbyte32(nw[k >> 2], k & 3);
            m_acc += msum;
            e_acc += e_here;
        }
    }
    if (colour == 1) block_add_pair(m_acc, e_acc, hist_slot);
}

// L % 64 != 0: one thread per 8-byte chunk (4 target sites, part of one plane word).
__global__ void int8_half_sweep_chunk8_kernel(int8_t* lat, int64_t L, uint64_t key, uint32_t t2, uint32_t t4, uint32_t all2,
                                       uint32_t all4, uint32_t sweep, int colour, int64_t* hist_slot)
{
    const int64_t G = L / 8;
    const int64_t chunks = L * G;
    if (colour == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        hist_slot[0] = 0;  // opened here, filled by the colour-1 pass of the same sweep
        hist_slot[1] = 0;
    }
    const PhiloxWordConsts pc = philox_consts(key, 0u, sweep, (uint32_t)colour);
    const uint32_t thr[2] = {t2, t4};
    const uint32_t zero2 = (t2 == 0u && all2 == 0u) ? ~0u : 0u, zero4 = (t4 == 0u && all4 == 0u) ? ~0u : 0u;
    long long m_acc = 0, e_acc = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < chunks;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / G, g = idx - i * G;
        const int64_t iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
        const int r = (int)((i + colour) & 1);
        int8_t* row = lat + i * L;
        const uint64_t cur = *reinterpret_cast<const uint64_t*>(row + 8 * g);
        const uint64_t upv = *reinterpret_cast<const uint64_t*>(lat + iu * L + 8 * g);
        const uint64_t dnv = *reinterpret_cast<const uint64_t*>(lat + id * L + 8 * g);
        // the one neighbour outside the chunk: column 8g-1 (r = 0) or 8g+8 (r = 1)
        const int64_t edge_col = r ? (g + 1 == G ? 0 : 8 * g + 8) : (g == 0 ? L - 1 : 8 * g - 1);
        const int edge = row[edge_col];

        // the chunk's 4 target sites have plane indices p0 .. p0+3 (p0 % 4 == 0), the
        // bits pos .. pos+3 of plane word p0 >> 5
        const uint64_t p0 = (uint64_t)i * (uint64_t)(L / 2) + 4ull * (uint64_t)g;
        const int pos = (int)(p0 & 31);
        const uint64_t qw = 8 * (p0 >> 5);
        const PhiloxWordConsts pcw =
            (qw >> 32) == 0 ? pc : philox_consts(key, (uint32_t)(qw >> 32), sweep, (uint32_t)colour);
        uint32_t alw = 0, h2m = 0, h4m = 0;
        for (int b = 0; b < 4; ++b) {
            const int k = 2 * b + r;
            const int s = sbyte(cur, k);
            const int left = k == 0 ? edge : sbyte(cur, k - 1);
            const int right = k == 7 ? edge : sbyte(cur, k + 1);
            const int h = s * (sbyte(upv, k) + sbyte(dnv, k) + left + right);
            alw |= (h <= 0 ? 1u : 0u) << (pos + b);
            h2m |= (h == 2 ? 1u : 0u) << (pos + b);
            h4m |= (h == 4 ? 1u : 0u) << (pos + b);
        }
        uint32_t lt[1] = {(h2m & all2) | (h4m & all4)};
        uint32_t und[1] = {(h2m & ~(all2 | zero2)) | (h4m & ~(all4 | zero4))};
        {
            const uint32_t sel[1] = {h2m}, ql[1] = {(uint32_t)qw};
            bitsliced_below<1, 2>(und, lt, sel, sel, ql, pcw, key, thr);
        }
        const uint32_t accm = alw | lt[0];

        uint64_t nv = cur;
        long long e_here = 0;
        for (int b = 0; b < 4; ++b) {
            const int k = 2 * b + r;  // byte of the target site in the chunk
            const int s = sbyte(cur, k);
            const int left = k == 0 ? edge : sbyte(cur, k - 1);
            const int right = k == 7 ? edge : sbyte(cur, k + 1);
            const int nn = sbyte(upv, k) + sbyte(dnv, k) + left + right;
            const bool acc = (accm >> (pos + b)) & 1u;
            const int snew = acc ? -s : s;
            if (acc) nv ^= (0xFEull << (8 * k));  // 0x01 <-> 0xFF
            e_here -= (long long)snew * nn;
        }
        if (nv != cur) *reinterpret_cast<uint64_t*>(row + 8 * g) = nv;
        if (colour == 1) {
            long long msum = 0;
            for (int k = 0; k < 8; ++k) msum += sbyte(nv, k);
            m_acc += msum;
            e_acc += e_here;
        }
    }
    if (colour == 1) block_add_pair(m_acc, e_acc, hist_slot);
}

__global__ void int8_observe_kernel(const int8_t* lat, int64_t L, int64_t* ME)
{
    long long m_acc = 0, e_acc = 0;
    const int64_t N = L * L;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / L, j = idx - i * L;
        const int s = lat[idx];
        m_acc += s;
        e_acc -= (long long)s * (lat[(i + 1 == L ? 0 : i + 1) * L + j] + lat[i * L + (j + 1 == L ? 0 : j + 1)]);
    }
    block_add_pair(m_acc, e_acc, ME);
}

__global__ void zero_pair_kernel(int64_t* p)
{
    p[0] = 0;
    p[1] = 0;
}

int grid_cap(int64_t work, int threads, int per_sm)
{
    const int64_t want = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_int8_init(int8_t* lat, int64_t L, uint64_t key, int start, cudaStream_t s)
{
    int8_init_kernel<<<grid_cap(L * (L / 8), 256, 16), 256, 0, s>>>(lat, L, key, start);
    return cudaGetLastError();
}

cudaError_t launch_int8_half_sweep(int8_t* lat, int64_t L, uint64_t key, uint32_t t2, uint32_t t4, uint32_t all2,
                                   uint32_t all4, uint32_t sweep, int colour, int64_t* hist_slot, cudaStream_t s)
{
    if (L % 64 == 0)
        int8_half_sweep_seg64_kernel<<<grid_cap(L * (L / 64), 256, 8), 256, 0, s>>>(lat, L, key, t2, t4, all2, all4,
                                                                                  sweep, colour, hist_slot);
    else
        int8_half_sweep_chunk8_kernel<<<grid_cap(L * (L / 8), 256, 8), 256, 0, s>>>(lat, L, key, t2, t4, all2, all4,
                                                                                   sweep, colour, hist_slot);
    return cudaGetLastError();
}

cudaError_t launch_int8_observe(const int8_t* lat, int64_t L, int64_t* ME, cudaStream_t s)
{
    zero_pair_kernel<<<1, 1, 0, s>>>(ME);
    int8_observe_kernel<<<grid_cap(L * L, 256, 8), 256, 0, s>>>(lat, L, ME);
    return cudaGetLastError();
}

}  // namespace ising

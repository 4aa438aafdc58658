// Resident sweep of one small bit-packed lattice: both colour planes stay in one
// CTA's shared memory for many sweeps, with a block barrier between half-sweeps
// instead of a kernel launch (the checkerboard schedule of Sec. 3.1).
#include "ising_internal.cuh"
#include "philox.cuh"
#include "word_update.cuh"

namespace ising {
namespace {

// Philox calls drawn side by side for every word with sites to test, before the
// rest are drawn one at a time (Sec. 3.1 acceptance on the bit planes of
// philox.cuh): a warp runs a call while any of its lanes needs it, and nearly every
// warp needs its words' first three, so drawing them together adds almost no issue
// slots and overlaps their latencies.
constexpr int kFirstCalls = 3;  // 9.2 flips/ns at L = 128 (8.9 with 2, 8.7 one call at a time)

// Resident form for one small lattice: both planes live in this CTA's shared
// memory for `nsweeps` sweeps, with a block barrier between half-sweeps instead
// of a kernel launch.  Same words, neighbours, draws and decisions as the tiled
// kernel; the white pass writes (M, E) of each sweep straight into the history.
template <int NT>
__global__ void __launch_bounds__(NT, 1) packed_resident_kernel(const __grid_constant__ LatticeDesc d, int nsweeps)
{
    extern __shared__ __align__(16) uint32_t planes_s[];
    __shared__ uint32_t red[2 * (NT / 32)];
    const int W = d.W, L = d.L;
    const int words = L * W;
    uint32_t* pl[2] = {planes_s, planes_s + words};
    const int tid = threadIdx.x;
    for (int k = tid; k < words; k += NT) {
        pl[0][k] = d.plane[0][k];
        pl[1][k] = d.plane[1][k];
    }
    __syncthreads();
    const uint64_t key = d.key;
    const bool q_small = L <= 131072;
    // thresholds 0 (never accept) are taken out of the test like 2^32 (always)
    const uint32_t zero2 = (d.t2 == 0u && d.all2 == 0u) ? ~0u : 0u, zero4 = (d.t4 == 0u && d.all4 == 0u) ? ~0u : 0u;
    const uint32_t thr[2] = {d.t2, d.t4};
    // the thresholds' bits in planes 0 .. 4 * kFirstCalls - 1 as all-ones / all-zero
    // masks, formed once per launch and held in registers (the opaque move keeps the
    // compiler from forming them again, from the launch-uniform thresholds, in every
    // plane of every half-sweep: six instructions a plane)
    constexpr int kPlanes = 4 * kFirstCalls;
    uint32_t K2[kPlanes], K4[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        K2[p] = 0u - ((d.t2 >> (31 - p)) & 1u);
        K4[p] = 0u - ((d.t4 >> (31 - p)) & 1u);
        asm volatile("mov.b32 %0, %0;" : "+r"(K2[p]));
        asm volatile("mov.b32 %0, %0;" : "+r"(K4[p]));
    }
    // (row, word) of idx = tid + k * NT, advanced without a division
    const int step_r = NT / W, step_w = NT - step_r * W;
    const int i_first = tid / W, w_first = tid - i_first * W;
    for (int s = 0; s < nsweeps; ++s) {
        const uint32_t sweep = d.sweep + (uint32_t)s;
        for (int colour = 0; colour < 2; ++colour) {
            const uint32_t* src = pl[colour ^ 1];
            uint32_t* tgt = pl[colour];
            const PhiloxWordConsts pc_all = philox_consts(key, 0u, sweep, (uint32_t)colour);
            uint32_t ups = 0, anti = 0;
            int i = i_first, w = w_first;
            for (int idx = tid; idx < words; idx += NT, i += step_r, w += step_w) {
                if (w >= W) {
                    w -= W;
                    ++i;
                }
                const int iu = i == 0 ? L - 1 : i - 1, id = i + 1 == L ? 0 : i + 1;
                const uint32_t up = src[iu * W + w], down = src[id * W + w], same = src[idx];
                uint32_t hz;
                if ((i + colour) & 1)
                    hz = __funnelshift_r(same, src[i * W + (w + 1 == W ? 0 : w + 1)], 1);
                else
                    hz = __funnelshift_l(src[i * W + (w == 0 ? W - 1 : w - 1)], same, 1);
                const uint64_t q0 = (uint64_t)i * (uint64_t)(L >> 3) + 8ull * (uint64_t)w;
                const PhiloxWordConsts pc =
                    q_small ? pc_all : philox_consts(key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
                const uint32_t tw = tgt[idx];
                uint32_t f[1], und[1], sel[1], anti0;
                classify_word(tw, up, down, same, hz, d.all2, d.all4, zero2, zero4, f[0], und[0], sel[0], anti0);
                if (und[0] != 0u) {
                    // calls 0 .. kFirstCalls-1 side by side, then one at a time while needed
                    uint32_t b[kFirstCalls], o[kFirstCalls][4];
#pragma unroll
                    for (int c = 0; c < kFirstCalls; ++c) b[c] = ((uint32_t)q0 ^ pc.x0k) ^ (uint32_t)c;
                    philox_calls<kFirstCalls>(b, 0u, pc, key, o);
#pragma unroll
                    for (int c = 0; c < kFirstCalls; ++c)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const uint32_t tm = (sel[0] & K2[4 * c + m]) | (~sel[0] & K4[4 * c + m]);
                            const uint32_t x = und[0] & (o[c][m] ^ tm);  // decided in this plane
                            f[0] |= x & tm;                             // ... below: U's bit 0, T's bit 1
                            und[0] &= ~x;
                        }
                    const uint32_t ql[1] = {(uint32_t)q0};
                    bitsliced_below<1, 2, kFirstCalls, 8>(und, f, sel, sel, ql, pc, key, thr);
                }
                if (colour == 1) {
                    ups += __popc(same);
                    anti += anti0 + 4u * __popc(f[0]) - 2u * __popc(f[0] & sel[0]);
                }
                tgt[idx] = tw ^ f[0];
                if (colour == 1) ups += __popc(tw ^ f[0]);
            }
            if (colour == 1) {
                const uint32_t u = __reduce_add_sync(0xffffffffu, ups);
                const uint32_t a = __reduce_add_sync(0xffffffffu, anti);
                if ((tid & 31) == 0) {
                    red[2 * (tid >> 5)] = u;
                    red[2 * (tid >> 5) + 1] = a;
                }
            }
            __syncthreads();
            if (colour == 1 && tid < 32) {
                // the warps' partial sums added by the first warp; a lattice of at most
                // 2^16 sites keeps every count far below 2^32
                const uint32_t u = tid < NT / 32 ? red[2 * tid] : 0u;
                const uint32_t a = tid < NT / 32 ? red[2 * tid + 1] : 0u;
                const uint32_t su = __reduce_add_sync(0xffffffffu, u);
                const uint32_t sa = __reduce_add_sync(0xffffffffu, a);
                if (tid == 0) {
                    const int64_t N = (int64_t)L * L;
                    d.hist[2 * (int64_t)sweep] = 2 * (int64_t)su - N;
                    d.hist[2 * (int64_t)sweep + 1] = 2 * (int64_t)sa - 2 * N;
                }
            }
        }
    }
    for (int k = tid; k < words; k += NT) {
        d.plane[0][k] = pl[0][k];
        d.plane[1][k] = pl[1][k];
    }
}

}  // namespace

int packed_resident_max_L() { return 256; }

cudaError_t launch_packed_resident(const LatticeDesc& d, int nsweeps, cudaStream_t s)
{
    // both planes: 2 * L * L/64 words, at most 8 KB for L <= 256 (within the default limit)
    const size_t smem = sizeof(uint32_t) * 2 * (size_t)d.L * (size_t)d.W;
    packed_resident_kernel<256><<<1, 256, smem, s>>>(d, nsweeps);
    return cudaGetLastError();
}

}  // namespace ising

// Device code of the three-dimensional checkerboard Metropolis sweep on bit-packed
// colour planes.
//
// The paper's Hamiltonian is written for a d-dimensional hypercubic lattice
// (Sec. 3) and its conclusion states that the checkerboard algorithm carries
// over to three dimensions; this file is that generalisation for the cubic
// L x L x L torus.  Every rule of the 2D sweep is kept (colour order black then
// white, h = sigma * nn, flip iff h <= 0 or U < T_h, integer thresholds, bit-plane
// Philox uniforms keyed by plane index); the neighbourhood has six sites, so the
// per-word neighbour count is a 6-input bitwise adder and three thresholds
// (h = 2, 4, 6) are tested.
//
// GB300 mapping: a persistent grid (two 256-thread CTAs per SM) walks groups of
// four adjacent words (one 16-byte vector load per neighbour row through the
// read-only path; 128 sites per thread iteration); words still undecided after
// two Philox calls finish from a per-warp queue in shared memory.  The kernel is bound by the
// integer pipes (Philox), not by memory: a half-sweep moves 3/16 byte per
// updated site, and the six neighbour rows of a word are re-read from L2.
//
// This header holds the kernel and everything it calls; it is compiled into the
// library (sweep3d.cu, thresholds read from the lattice's descriptor) and, at run
// time, for one lattice's thresholds as compile-time constants (jit.cu, with NVRTC),
// so it includes only headers NVRTC can compile.
#pragma once
#include "ising_device.cuh"
#include "word_update.cuh"

namespace ising {
namespace cubic {

// Thresholds of the acceptance test (h = 2, 4, 6): read from the descriptor, or
// compile-time constants of a kernel compiled for one temperature (the 2D sweep's
// FixedThresholds, with three thresholds).
struct RuntimeThresholds3 {
    static constexpr bool kFixed = false;
    static constexpr uint32_t t2 = 0u, t4 = 0u, t6 = 0u, all2 = 0u, all4 = 0u, all6 = 0u;
};
template <uint32_t T2, uint32_t T4, uint32_t T6, uint32_t ALL2, uint32_t ALL4, uint32_t ALL6>
struct FixedThresholds3 {
    static constexpr bool kFixed = true;
    static constexpr uint32_t t2 = T2, t4 = T4, t6 = T6, all2 = ALL2, all4 = ALL4, all6 = ALL6;
};

// Classes of one 32-site target word t from its six neighbour words: f = sites
// that flip without a test (h <= 0, or a threshold of 2^32), und = sites to test
// against T2 (selA, h = 2), T4 (selB, h = 4) or T6 (the rest, h = 6); zeroN = ~0u
// for a threshold of 0 (never accept).  The fused observables come from the adder
// bits as in 2D (word_update.cuh): a site with n anti-aligned neighbours has n if
// it stays and 6 - n if it flips.  Sites with n >= 3 always flip, so anti0 = the
// sum of n minus the always-flipped sites' 2 (b0) + 4 (b1) + 8 (b2) parts, and
// once the word is decided the flip mask f adds 6 popc(f) - 2 popc(f & selB) -
// 4 popc(f & selA) (the tested classes n = 1 and n = 2 among the flipped sites).
__device__ __forceinline__ void classify_word3d(uint32_t t, uint32_t up, uint32_t dn, uint32_t no, uint32_t so,
                                                uint32_t same, uint32_t hz, uint32_t all2, uint32_t all4,
                                                uint32_t all6, uint32_t zero2, uint32_t zero4, uint32_t zero6,
                                                uint32_t& f, uint32_t& und, uint32_t& selA, uint32_t& selB,
                                                uint32_t& anti0)
{
    // anti-aligned neighbour bits and their 6-input sum n = 4*b2 + 2*b1 + b0: two
    // full adders over three inputs each, then the sum bits added (b0, carry c3)
    // and the three weight-2 carries added (b1, b2)
    const uint32_t a0 = t ^ up, a1 = t ^ dn, a2 = t ^ no;
    const uint32_t a3 = t ^ so, a4 = t ^ same, a5 = t ^ hz;
    const uint32_t s1 = a0 ^ a1 ^ a2, c1 = (a0 & a1) | (a2 & (a0 ^ a1));
    const uint32_t s2 = a3 ^ a4 ^ a5, c2 = (a3 & a4) | (a5 & (a3 ^ a4));
    const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t b1 = c1 ^ c2 ^ c3;
    const uint32_t b2 = (c1 & c2) | (c3 & (c1 ^ c2));
    // h = 6 - 2n: n >= 3 (h <= 0) always; n = 2 (h = 2): U < T2; n = 1 (h = 4):
    // U < T4; n = 0 (h = 6): U < T6
    const uint32_t always = b2 | (b1 & b0);
    const uint32_t h2 = b1 & ~b0 & ~b2, h4 = b0 & ~b1 & ~b2, h6 = ~(b0 | b1 | b2);
    f = always | (h2 & all2) | (h4 & all4) | (h6 & all6);
    und = (h2 & ~(all2 | zero2)) | (h4 & ~(all4 | zero4)) | (h6 & ~(all6 | zero6));
    selA = h2;
    selB = h4;
    anti0 = __popc(b0) + 2u * __popc(b1) - 4u * __popc(b2) - 2u * __popc(b0 & (b1 | b2)) - 4u * __popc(b1 & (b0 | b2));
}

// Words still undecided after the first two Philox calls wait in a per-warp queue;
// an entry is two 16-byte slots: (position low, position high, undecided sites,
// flips so far) and (h = 2 sites, h = 4 sites, old target word, unused).  The
// queue is checked (and drained 32 at a time while it holds 32) once per group of
// four words, so it takes 31 + 4 * 32 entries (40 KB of static shared memory per
// 256-thread CTA); checking once per group keeps the drain inlined at one place.
constexpr int kQueueCap3 = 160;

// Calls 2..7 for the top n queue entries, one per lane < n (every lane of the warp
// takes part), then the words' final values and, with COUNT, their counts.
template <bool COUNT, typename TH>
__device__ __forceinline__ void drain_queue3d(const CubicDesc& d, uint32_t* tgt, const PhiloxWordConsts& pc_all,
                                              bool q_small, int colour, uint32_t sweep, uint4* wq, int& qn, int n,
                                              int lane, uint32_t& ups, uint32_t& anti)
{
    const bool act = lane < n;
    uint4 e0 = make_uint4(0u, 0u, 0u, 0u), e1 = make_uint4(0u, 0u, 0u, 0u);
    if (act) {
        e0 = wq[2 * (qn - n + lane)];
        e1 = wq[2 * (qn - n + lane) + 1];
    }
    qn -= n;
    __syncwarp();  // entries read before the next pushes overwrite them
    const uint64_t pos = (uint64_t)e0.x | ((uint64_t)e0.y << 32);
    uint32_t und[1] = {e0.z}, f[1] = {e0.w};
    const uint32_t selA[1] = {e1.x}, selB[1] = {e1.y};
    const uint64_t q = 8ull * pos;
    const uint32_t ql[1] = {(uint32_t)q};
    const PhiloxWordConsts pc = q_small ? pc_all : philox_consts(d.key, (uint32_t)(q >> 32), sweep, (uint32_t)colour);
    const uint32_t thr[3] = {TH::kFixed ? TH::t2 : d.t2, TH::kFixed ? TH::t4 : d.t4, TH::kFixed ? TH::t6 : d.t6};
    bitsliced_below<1, 3, 2, 8, true>(und, f, selA, selB, ql, pc, d.key, thr);
    if (act) {
        const uint32_t nw = e1.z ^ f[0];
        tgt[pos] = nw;
        if (COUNT) {
            ups += __popc(nw);
            anti += 6u * __popc(f[0]) - 2u * __popc(f[0] & selB[0]) - 4u * __popc(f[0] & selA[0]);
        }
    }
}

template <int G>
__device__ __forceinline__ void load_ro(const uint32_t* p, uint32_t v[G])
{
    if constexpr (G == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = __ldg(p + k);
    }
}

// The source-colour neighbours of G adjacent target words (w .. w+G-1) of row
// (i, j): rows (i+-1, j) and (i, j+-1) at the same words, and the row's own
// source words, same (bit b <-> same m) and hz (bit b <-> m - 1 or m + 1).
template <int G>
struct Nbr {
    uint32_t up[G], dn[G], no[G], so[G], sm[G], hz[G];
};

template <int G>
__device__ __forceinline__ void load_neighbours(const uint32_t* __restrict__ src, int64_t L, int W, int64_t i,
                                                int64_t j, int w, int par, Nbr<G>& n)
{
    const int64_t im = (i == 0) ? L - 1 : i - 1, ip = (i == L - 1) ? 0 : i + 1;
    const int64_t jm = (j == 0) ? L - 1 : j - 1, jp = (j == L - 1) ? 0 : j + 1;
    const uint32_t* row = src + (i * L + j) * W;
    load_ro<G>(src + (im * L + j) * W + w, n.up);
    load_ro<G>(src + (ip * L + j) * W + w, n.dn);
    load_ro<G>(src + (i * L + jm) * W + w, n.no);
    load_ro<G>(src + (i * L + jp) * W + w, n.so);
    load_ro<G>(row + w, n.sm);
    if (par) {  // target at odd k: z-neighbours at source m and m + 1
        const uint32_t next = __ldg(row + ((w + G == W) ? 0 : w + G));
#pragma unroll
        for (int k = 0; k < G; ++k) n.hz[k] = __funnelshift_r(n.sm[k], k + 1 < G ? n.sm[k + 1] : next, 1);
    } else {  // target at even k: z-neighbours at source m - 1 and m
        const uint32_t prev = __ldg(row + ((w == 0) ? W - 1 : w - 1));
#pragma unroll
        for (int k = 0; k < G; ++k) n.hz[k] = __funnelshift_l(k > 0 ? n.sm[k - 1] : prev, n.sm[k], 1);
    }
}

// The same from the word offsets of the five source rows (row, i-1, i+1, j-1, j+1).
template <int G>
__device__ __forceinline__ void load_neighbours_at(const uint32_t* __restrict__ src, int W, int64_t row,
                                                   int64_t up, int64_t dn, int64_t no, int64_t so, int w, int par,
                                                   Nbr<G>& n)
{
    const uint32_t* rp = src + row;
    load_ro<G>(src + up + w, n.up);
    load_ro<G>(src + dn + w, n.dn);
    load_ro<G>(src + no + w, n.no);
    load_ro<G>(src + so + w, n.so);
    load_ro<G>(rp + w, n.sm);
    if (par) {
        const uint32_t next = __ldg(rp + ((w + G == W) ? 0 : w + G));
#pragma unroll
        for (int k = 0; k < G; ++k) n.hz[k] = __funnelshift_r(n.sm[k], k + 1 < G ? n.sm[k + 1] : next, 1);
    } else {
        const uint32_t prev = __ldg(rp + ((w == 0) ? W - 1 : w - 1));
#pragma unroll
        for (int k = 0; k < G; ++k) n.hz[k] = __funnelshift_l(k > 0 ? n.sm[k - 1] : prev, n.sm[k], 1);
    }
}

// Block sum of two per-thread counts, then 2x the sums added to out[0..1].
template <int NT>
__device__ __forceinline__ void block_add_twice(unsigned long long a, unsigned long long b,
                                                unsigned long long* red, int64_t* out)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sa = 0, sb = 0;
        for (int k = 0; k < NT / 32; ++k) {
            sa += red[2 * k];
            sb += red[2 * k + 1];
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(out), 2ull * sa);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 1), 2ull * sb);
    }
}

// Each word draws its first two Philox calls (8 bit planes) in step with its warp;
// words with sites left wait in the warp's queue and are finished 32 at a time,
// one per lane (the 2D tile routine does the same).  A queued word is stored twice:
// as far as decided, then final (ordered by __syncwarp).  COUNT (the colour-1 pass)
// adds the fused observables; as a template parameter it leaves the colour-0 pass
// without their instructions.
//
// Work order: each warp takes the next 8 x 32 word groups (rows in plane order) from
// the counter work[colour] and its lanes walk them 32 consecutive groups at a time.
// So the groups in flight always form one narrow band that moves through the plane,
// and the source rows of slices i - 1 and i + 1 are read while they are still in L2
// (with a fixed grid-stride split the CTAs drift apart over a half-sweep and a row
// loaded for slice i - 1 is evicted before slice i + 1 needs it).  work[colour] is zero
// at launch: the launch of the other colour, which runs before it on the stream,
// clears it (and this launch clears work[colour ^ 1] for the next one).
template <int NT, int G, bool COUNT, typename TH = RuntimeThresholds3>
__global__ void __launch_bounds__(NT, 2) cubic_half_sweep_kernel(const __grid_constant__ CubicDesc d, int colour,
                                                                 uint32_t sweep, unsigned long long* work)
{
    __shared__ unsigned long long red[2 * (NT / 32)];
    __shared__ uint4 queues[(NT / 32) * 2 * kQueueCap3];
    const int64_t L = d.L;
    const int W = d.W, WG = W / G;
    const int64_t ngroups = L * L * WG;
    const uint32_t* __restrict__ src = d.plane[colour ^ 1];
    uint32_t* __restrict__ tgt = d.plane[colour];
    const int lane = threadIdx.x & 31;
    uint4* wq = queues + (threadIdx.x >> 5) * 2 * kQueueCap3;
    int qn = 0;  // entries in the warp's queue (the same in every lane)
    if (colour == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        // open this sweep's (M, E) slot: M = 2 * ups - N, E = 2 * anti - 3N
        const int64_t N = L * L * L;
        d.hist[2 * (int64_t)sweep] = -N;
        d.hist[2 * (int64_t)sweep + 1] = -3 * N;
    }
    const bool q_small = cubic_q_small(L);
    const PhiloxWordConsts pc_all = philox_consts(d.key, 0u, sweep, (uint32_t)colour);
    // thresholds and their always / never masks: constants of a fixed-threshold build
    const uint32_t t2 = TH::kFixed ? TH::t2 : d.t2, t4 = TH::kFixed ? TH::t4 : d.t4, t6 = TH::kFixed ? TH::t6 : d.t6;
    const uint32_t all2 = TH::kFixed ? TH::all2 : d.all2, all4 = TH::kFixed ? TH::all4 : d.all4;
    const uint32_t all6 = TH::kFixed ? TH::all6 : d.all6;
    const uint32_t zero2 = (t2 == 0u && all2 == 0u) ? ~0u : 0u;
    const uint32_t zero4 = (t4 == 0u && all4 == 0u) ? ~0u : 0u;
    const uint32_t zero6 = (t6 == 0u && all6 == 0u) ? ~0u : 0u;
    const uint32_t thr[3] = {t2, t4, t6};
    // per-thread counts stay below 2^31 in magnitude: even a whole warp sees at most
    // L^3 / (2 * 152 * 2 * 8) white sites (< 1.2e8 at L = 8192) with at most 7
    // counted bits each
    uint32_t ups = 0, anti = 0;
    // (i, j, word group) of a lane's group, advanced by 32 groups per step without
    // divisions: step_w groups within a row plus step_r rows, step_r = step_i * L + step_j
    constexpr int kSteps = 8;
    const int64_t stride = 32;
    const int64_t step_r = stride / WG;
    const int step_w = (int)(stride - step_r * WG);
    const int64_t step_i = step_r / L, step_j = step_r - step_i * L;
    int64_t i = 0, j = 0;
    int wg = 0;
    // word offset of row (i, j), carried along the walk, and the offsets from it to
    // the rows (i-+1, j) and (i, j-+1) away from / across the torus seam
    const int64_t Wl = W, LW = L * Wl, LLW = L * LW;
    const int64_t step_off = step_r * Wl;
    int64_t row = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) work[colour ^ 1] = 0ull;
    for (;;) {
        unsigned long long taken = 0ull;
        if (lane == 0) taken = atomicAdd(work + colour, 32ull * kSteps);
        const int64_t base = (int64_t)__shfl_sync(0xffffffffu, taken, 0);
        if (base >= ngroups) break;
        {
            const int64_t r0 = (base + lane) / WG;
            wg = (int)(base + lane - r0 * WG);
            i = r0 / L;
            j = r0 - i * L;
            row = r0 * Wl;
        }
        // every lane runs every step (the votes and the queue need the whole warp); a
        // lane past the end works on group 0 and keeps nothing
        for (int s = 0; s < kSteps; ++s) {
            const int64_t g0 = base + 32 * s;
            if (g0 >= ngroups) break;
            const bool valid = g0 + lane < ngroups;
            const int64_t vi = valid ? i : 0, vj = valid ? j : 0, vrow = valid ? row : 0;
            const int w = valid ? wg * G : 0;
            const int par = (int)((vi + vj + colour) & 1);
            const int64_t up = vrow + (vi == 0 ? LLW - LW : -LW), dn = vrow + (vi == L - 1 ? LW - LLW : LW);
            const int64_t no = vrow + (vj == 0 ? LW - Wl : -Wl), so = vrow + (vj == L - 1 ? Wl - LW : Wl);
            Nbr<G> n;
            load_neighbours_at<G>(src, W, vrow, up, dn, no, so, w, par, n);
            uint32_t* trow = tgt + vrow + w;
            uint32_t t[G];
            if constexpr (G == 4) {
                const uint4 q = *reinterpret_cast<const uint4*>(trow);
                t[0] = q.x;
                t[1] = q.y;
                t[2] = q.z;
                t[3] = q.w;
            } else {
    #pragma unroll
                for (int k = 0; k < G; ++k) t[k] = trow[k];
            }
            // q0 = r * (L/8) + 8w = 8 * (row + w) with L/8 = 8W; it is a multiple of 8 * G,
            // so the group's calls q0 .. q0 + 8G - 1 share q's high word
            const uint64_t q0 = 8ull * (uint64_t)(vrow + w);
            const PhiloxWordConsts pc =
                q_small ? pc_all : philox_consts(d.key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
            uint32_t f[G], und[G], selA[G], selB[G], ql[G];
    #pragma unroll
            for (int k = 0; k < G; ++k) {
                uint32_t anti0;
                classify_word3d(t[k], n.up[k], n.dn[k], n.no[k], n.so[k], n.sm[k], n.hz[k], all2, all4, all6, zero2,
                                zero4, zero6, f[k], und[k], selA[k], selB[k], anti0);
                if (!valid) und[k] = 0u;
                if (COUNT && valid) {
                    ups += __popc(n.sm[k]);
                    anti += anti0;
                }
                ql[k] = (uint32_t)q0 + 8u * k;
            }
            // calls 0-1: nearly every warp needs both, so both are drawn without a vote
            bitsliced_below<G, 3, 0, 2, true, false>(und, f, selA, selB, ql, pc, d.key, thr);
            uint32_t nw[G];
    #pragma unroll
            for (int k = 0; k < G; ++k) nw[k] = t[k] ^ f[k];
            if (valid) {
                if constexpr (G == 4) {
                    *reinterpret_cast<uint4*>(trow) = make_uint4(nw[0], nw[1], nw[2], nw[3]);
                } else {
    #pragma unroll
                    for (int k = 0; k < G; ++k) trow[k] = nw[k];
                }
            }
    #pragma unroll
            for (int k = 0; k < G; ++k) {
                const bool pend = und[k] != 0u;
                if (COUNT && valid && !pend) {
                    ups += __popc(nw[k]);
                    anti += 6u * __popc(f[k]) - 2u * __popc(f[k] & selB[k]) - 4u * __popc(f[k] & selA[k]);
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, pend);
                if (pend) {
                    const int slot = qn + __popc(bal & ((1u << lane) - 1u));
                    const uint64_t pos = (uint64_t)(vrow + w + k);
                    wq[2 * slot] = make_uint4((uint32_t)pos, (uint32_t)(pos >> 32), und[k], f[k]);
                    wq[2 * slot + 1] = make_uint4(selA[k], selB[k], t[k], 0u);
                }
                qn += __popc(bal);
            }
            if (qn >= 32) {
                __syncwarp();  // pushes visible to the draining lanes
                do {
                    drain_queue3d<COUNT, TH>(d, tgt, pc_all, q_small, colour, sweep, wq, qn, 32, lane, ups, anti);
                } while (qn >= 32);
            }
            wg += step_w;
            j += step_j;
            i += step_i;
            row += step_off;
            if (wg >= WG) {
                wg -= WG;
                ++j;
                row += Wl;
            }
            if (j >= L) {
                j -= L;
                ++i;
            }
        }
    }
    if (qn > 0) {
        __syncwarp();
        drain_queue3d<COUNT, TH>(d, tgt, pc_all, q_small, colour, sweep, wq, qn, qn, lane, ups, anti);
    }
    // a lane's bond count may be negative (a word's negative part can be added by
    // the lane that queued it and the rest by the lane that drained it), so it is
    // widened as a signed value; the block's total is not negative
    if (COUNT)
        block_add_twice<NT>(ups, (unsigned long long)(long long)(int32_t)anti, red, d.hist + 2 * (int64_t)sweep);
}

}  // namespace cubic
}  // namespace ising

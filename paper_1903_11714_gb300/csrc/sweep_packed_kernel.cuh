// Device code of the bit-packed checkerboard half-sweep (the paper's UpdateOptim, Algorithm 2, on
// multi-spin-coded colour planes) with fused magnetisation / energy counts.
//
// Layout: two planes (black = colour 0, white = colour 1), L rows of W = L/64
// 32-bit words each; bit b of word w in row i of plane c is the site
// (i, j = 2(32w + b) + ((i + c) & 1)), bit 1 = spin +1.
//
// Neighbours of a target site (i, 2k + r), r = (i + c) & 1, all in the other
// plane: (i-1, k), (i+1, k), (i, k), and (i, k-1) when r = 0 or (i, k+1) when
// r = 1 (torus wrap in both directions).  This is the neighbour topology of the
// compact sub-lattice formulas in Sec. 3.2, with the boundary compensation of
// Algorithms 1-2 replaced by halo rows and a wrapped funnel shift.
//
// Per 32-site word: n_anti (number of anti-aligned neighbours, 0..4) comes from a
// bitwise 4-input adder; h = sigma * nn = 4 - 2 n_anti.  h <= 0 flips always;
// h = 2 flips iff the site's uniform U is below T2, h = 4 iff below T4 (Sec. 3.1
// acceptance min{1, exp(-2 beta h)} as an integer threshold), with U compared bit
// plane by bit plane on whole words (word_update.cuh).  Each word draws two Philox
// calls in step with its warp; the ~10 % of words with sites still undecided
// after them finish from a per-warp queue (update_tile).
//
// Each persistent CTA walks the tile table: a tile is `tile_rows` full rows of
// one lattice.  A tile's source rows (plus the halo rows above and below, wrapped)
// and target rows are staged into shared memory with bulk async copies
// (cp.async.bulk, completion on an mbarrier), double-buffered so the next tile
// lands while the current one is computed.  There is no CTA-wide barrier per tile:
// each warp counts itself out of a stage when it is done with it, and the last warp
// out issues the copies of the stage's next tile, so warps run up to a tile apart
// instead of waiting for the slowest at every tile.
//
// This header holds the kernel and everything it calls; it is compiled into the
// library (sweep_packed.cu, thresholds read from each lattice's descriptor) and,
// at run time, for one lattice's thresholds as compile-time constants (jit.cu,
// with NVRTC), so it includes only headers NVRTC can compile.
#pragma once
#include "ising_device.cuh"
#include "philox.cuh"
#include "word_update.cuh"

// Threads per SM the register allocation must leave room for (a CTA of NT
// threads gets a register cap of 65536 / ISING_SWEEP_THREADS_PER_SM per thread).
#ifndef ISING_SWEEP_THREADS_PER_SM
#define ISING_SWEEP_THREADS_PER_SM 512
#endif

namespace ising {
namespace sweep {


__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// A 16-byte shared-memory load the compiler may not merge with an earlier one (so a
// value read before a long computation is read again instead of held in registers).
__device__ __forceinline__ uint4 ld_shared_v4(const uint32_t* p)
{
    uint4 v;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Bounded wait: returns false after `limit` SM clocks without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Lattice owning global tile t (binary search of the prefix table).
__device__ __forceinline__ int lattice_of_tile(const int32_t* tile_start, int count, int t)
{
    int lo = 0, hi = count;  // tile_start[lo] <= t < tile_start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_start + mid) <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

struct TileInfo {
    int lat;
    bool live;
};

// Descriptor of lattice `lat`: from the device table, or -- for a launch over a
// single lattice (ONE) -- from the kernel parameter, whose fields are then
// launch-uniform operands (round keys, thresholds) instead of per-thread loads.
template <bool ONE>
__device__ __forceinline__ const LatticeDesc& desc_at(const TileTable& tt, const LatticeDesc& one, int lat)
{
    if constexpr (ONE)
        return one;
    else
        return tt.desc[lat];
}

template <bool ONE>
__device__ __forceinline__ TileInfo tile_info(const TileTable& tt, const LatticeDesc& one, int count, int t,
                                              int step)
{
    TileInfo ti;
    ti.lat = ONE ? 0 : lattice_of_tile(tt.tile_start, count, t);
    const LatticeDesc& d = desc_at<ONE>(tt, one, ti.lat);
    ti.live = d.active && (d.sweep + (uint32_t)step < d.target);
    return ti;
}

template <bool ONE>
__device__ __forceinline__ int tile_base(const TileTable& tt, int lat)
{
    if constexpr (ONE)
        return 0;
    else
        return __ldg(tt.tile_start + lat);
}

// One thread (thread 0 for the first two tiles, afterwards lane 0 of the last warp to
// release the stage) stages the tile's rows.  Source rows [i0 - HB, i0 + TR + HB) (wrapped)
// and target rows [i0, i0 + TR).  Every copy starts on a 16-byte boundary: with
// W % 4 == 0 every row does (TR may then be 2); otherwise HB = 4 and tiles start
// on rows that are multiples of 4, so each copied block starts at a multiple of
// 4 rows.
//
// Column blocks (tile_words = CW < W, W % 4 == 0, HB = 1): tile (row block rb, column
// block cb) covers rows i0 = rb * TR .. and words w0 = cb * CW .. w0 + CW - 1.  Each
// source row is staged as words w0 - 4 .. w0 + CW + 3 (CW + 8 words; the 4 words on
// either side, wrapped round the row at its ends, give the horizontal neighbours of
// the block's edge words), each target row as its CW words.  All copies are whole
// 16-byte units at 16-byte boundaries.
//
// TILES: 0 = whole rows only, 1 = column blocks only, 2 = either (decided per lattice).
template <int TILES>
__device__ __forceinline__ void issue_tile(const LatticeDesc& d, int local_tile, int colour, uint32_t* stage,
                                           uint64_t* bar, uint32_t extra_tx)
{
    const int W = d.W, L = d.L, TR = d.tile_rows, HB = d.halo_rows, CW = d.tile_words ? d.tile_words : W;
    if (TILES != 0 && (TILES == 1 || CW != W)) {
        const int ncb = W / CW;
        const int rb = local_tile / ncb, cb = local_tile - rb * ncb;
        const int i0 = rb * TR, w0 = cb * CW, SW = CW + 8;
        const uint32_t* src = d.plane[colour ^ 1];
        const uint32_t* tgt = d.plane[colour];
        uint32_t* s_src = stage;
        uint32_t* s_tgt = stage + (size_t)(TR + 2 * HB) * SW;
        mbar_expect_tx(bar, 4u * (uint32_t)((TR + 2 * HB) * SW + TR * CW) + extra_tx);
        for (int a = 0; a < TR + 2 * HB; ++a) {
            int row = i0 - HB + a;
            if (row < 0) row += L;
            if (row >= L) row -= L;
            const uint32_t* rp = src + (size_t)row * W;
            uint32_t* dst = s_src + (size_t)a * SW;
            if (w0 == 0) {
                bulk_copy_g2s(dst, rp + W - 4, 16u, bar);
                bulk_copy_g2s(dst + 4, rp, 4u * (uint32_t)(CW + 4), bar);
            } else if (w0 + CW == W) {
                bulk_copy_g2s(dst, rp + w0 - 4, 4u * (uint32_t)(CW + 4), bar);
                bulk_copy_g2s(dst + CW + 4, rp, 16u, bar);
            } else {
                bulk_copy_g2s(dst, rp + w0 - 4, 4u * (uint32_t)SW, bar);
            }
        }
        for (int a = 0; a < TR; ++a)
            bulk_copy_g2s(s_tgt + (size_t)a * CW, tgt + (size_t)(i0 + a) * W + w0, 4u * (uint32_t)CW, bar);
        return;
    }
    const int i0 = local_tile * TR;
    const uint32_t* src = d.plane[colour ^ 1];
    const uint32_t* tgt = d.plane[colour];
    const uint32_t row_bytes = (uint32_t)W * 4u;
    int ia = i0 - HB;
    if (ia < 0) ia += L;
    int ib = i0 + TR;
    if (ib >= L) ib -= L;
    uint32_t* s_src = stage;
    uint32_t* s_tgt = stage + (size_t)(TR + 2 * HB) * W;
    mbar_expect_tx(bar, row_bytes * (uint32_t)(2 * HB + 2 * TR) + extra_tx);
    bulk_copy_g2s(s_src, src + (size_t)ia * W, row_bytes * HB, bar);
    bulk_copy_g2s(s_src + (size_t)HB * W, src + (size_t)i0 * W, row_bytes * TR, bar);
    bulk_copy_g2s(s_src + (size_t)(HB + TR) * W, src + (size_t)ib * W, row_bytes * HB, bar);
    bulk_copy_g2s(s_tgt, tgt + (size_t)i0 * W, row_bytes * TR, bar);
}

template <int G>
__device__ __forceinline__ void load_group(const uint32_t* p, uint32_t v[G])
{
    if constexpr (G == 4) {
        const uint4 q = *reinterpret_cast<const uint4*>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else if constexpr (G == 2) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = *p;
    }
}

template <int G>
__device__ __forceinline__ void store_group(uint32_t* p, const uint32_t v[G])
{
    if constexpr (G == 4)
        *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
    else if constexpr (G == 2)
        *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
    else
        *p = v[0];
}

// Entries of the per-warp queue of words still undecided after the first two
// Philox calls: (word position in the tile, undecided sites, flips so far, h = 2
// sites).  The queue is checked (and drained 32 at a time while it holds 32) once
// per group of words in CTAs of up to 256 threads, so it must take 31 + 4 * 32
// entries; 512-thread CTAs check it after every two words and take 31 + 2 * 32, so
// that two 100 KB tile stages and the queues still fit one CTA's shared memory.
__host__ __device__ constexpr int queue_cap(int threads) { return threads <= 256 ? 160 : 96; }

// Thresholds of the acceptance test.  RuntimeThresholds: read from the lattice's
// descriptor, one kernel for every temperature.  FixedThresholds: compile-time
// constants of a kernel compiled for one lattice's temperature (at run time, by
// jit.cu), so that each bit plane's comparison is folded to the logic its two
// threshold bits need (one to three operations instead of four); the decisions are
// the same bit for bit.  ALL = ~0u where the threshold is 2^32 (accept always).
struct RuntimeThresholds {
    static constexpr bool kFixed = false;
    static constexpr uint32_t t2 = 0u, t4 = 0u, all2 = 0u, all4 = 0u;
};
template <uint32_t T2, uint32_t T4, uint32_t ALL2, uint32_t ALL4>
struct FixedThresholds {
    static constexpr bool kFixed = true;
    static constexpr uint32_t t2 = T2, t4 = T4, all2 = ALL2, all4 = ALL4;
};

// Per-tile constants of the word update.  A tile is TR rows of CW words (CW = W:
// whole rows; else a column block starting at word w0).
struct TileCtx {
    const uint32_t* s_src;  // source rows i0 - HB .. i0 + TR + HB - 1 (shared memory), SW words apart
    const uint32_t* s_tgt;  // target rows i0 .. i0 + TR - 1 (shared memory), CW words apart
    uint32_t* out;          // target plane at (row i0, word w0) (global memory)
    uint64_t q_tile;        // Philox call index of the tile's first word: 8 * (i0 * W + w0)
    uint64_t key;
    uint32_t sweep, t2, t4, all2, all4, zero2, zero4;
    int W, HB, colour;
    int CW, SW;             // words per tile row; smem source row stride (CW + 8 for column
                            // blocks, whose rows start with 4 halo words; W for whole rows)
    int par0;               // (i0 + colour) & 1: row i0 + r has its horizontal neighbour on the right iff r + par0 is odd
    bool q_small;           // every call index of the lattice below 2^32
};

__device__ __forceinline__ PhiloxWordConsts group_consts(const TileCtx& x, const PhiloxWordConsts& pc_tile, uint64_t q)
{
    return x.q_small ? pc_tile : philox_consts(x.key, (uint32_t)(q >> 32), x.sweep, (uint32_t)x.colour);
}

// Calls 2..7 for the top n queue entries, one per lane < n (every lane of the warp
// takes part), then the words' final values and, with COUNT, their counts.  An entry's
// first field is (row in the tile) << 16 | (word in the tile row).
template <bool COUNT, bool BLOCKS, typename TH>
__device__ __forceinline__ void drain_queue(const TileCtx& x, const PhiloxWordConsts& pc_tile, uint4* wq, int& qn,
                                            int n, int lane, uint32_t& ups, uint32_t& anti)
{
    const bool act = lane < n;
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (act) e = wq[qn - n + lane];
    qn -= n;
    __syncwarp();  // entries read before the next pushes overwrite them
    uint32_t und[1] = {e.y}, fm[1] = {e.z};
    const uint32_t sel[1] = {e.w};
    // whole rows: the entry holds the word's offset from the tile's first word (the same
    // in the plane and in shared memory); column blocks: (row << 16) | word in the row
    const uint32_t er = e.x >> 16, ew = e.x & 0xFFFFu;
    const uint32_t off = BLOCKS ? er * (uint32_t)x.W + ew : e.x;
    const uint64_t q = x.q_tile + 8ull * off;
    const uint32_t ql[1] = {(uint32_t)q};
    const uint32_t thr[2] = {TH::kFixed ? TH::t2 : x.t2, TH::kFixed ? TH::t4 : x.t4};
    bitsliced_below<1, 2, 2, 8, true>(und, fm, sel, sel, ql, group_consts(x, pc_tile, q), x.key, thr);
    if (act) {
        const uint32_t nw = x.s_tgt[BLOCKS ? er * (uint32_t)x.CW + ew : e.x] ^ fm[0];
        x.out[off] = nw;
        if (COUNT) {
            ups += __popc(nw);
            anti += 4u * __popc(fm[0]) - 2u * __popc(fm[0] & sel[0]);
        }
    }
}

// One staged tile of TR rows, G adjacent words per thread and step (G = 4 when
// W % 4 == 0: one 128-bit shared-memory load per neighbour row).  Every word
// draws its first two Philox calls (8 bit planes, which decide all of a word's
// sites with probability about 0.9 at the critical point) in step with its warp;
// words with sites left wait in the warp's queue, drained 32 at a time with one
// word per lane.  So the rare long comparisons no longer hold a whole warp, which
// draws about 2.2 calls per word instead of the ~3.4 a warp-wide early exit needs.
// A queued word is stored twice: as far as decided, then final (ordered by
// __syncwarp).  With COUNT (the colour-1 pass) the fused M/E counts are added (the
// bond count from the adder bits, derived in word_update.cuh); COUNT is a template
// parameter so that the colour-0 pass carries none of their
// instructions (predicated, they cost ~9 % of its issue slots).
//
// BLOCKS: the tile is a column block (its source rows carry halo words, so the
// horizontal neighbours need no wrap); else whole rows (CW = SW = W, wrapped).
template <int NT, int G, bool COUNT, bool BLOCKS, typename TH, bool INPLACE = false>
__device__ __forceinline__ void update_tile(const TileCtx& x, const PhiloxWordConsts& pc_tile, int nwords, uint4* wq,
                                            uint32_t& ups, uint32_t& anti)
{
    // thresholds and their always / never masks: constants of a fixed-threshold build
    const uint32_t t2 = TH::kFixed ? TH::t2 : x.t2, t4 = TH::kFixed ? TH::t4 : x.t4;
    const uint32_t all2 = TH::kFixed ? TH::all2 : x.all2, all4 = TH::kFixed ? TH::all4 : x.all4;
    const uint32_t zero2 = TH::kFixed ? ((TH::t2 == 0u && TH::all2 == 0u) ? ~0u : 0u) : x.zero2;
    const uint32_t zero4 = TH::kFixed ? ((TH::t4 == 0u && TH::all4 == 0u) ? ~0u : 0u) : x.zero4;
    const int tid = threadIdx.x, lane = tid & 31;
    const int W = x.W, CW = BLOCKS ? x.CW : W, SW = BLOCKS ? x.SW : W, WG = CW / G, ngroups = nwords / G;
    int qn = 0;  // entries in the warp's queue (the same in every lane)
    // (row, group) of g = tid + k*NT, advanced without a division
    const int step_r = NT / WG, step_w = NT - step_r * WG;
    int r = tid / WG, wg = tid - r * WG;
    for (int k0 = 0; k0 < ngroups; k0 += NT) {
        // every lane runs every step (the votes and the queue need the whole warp);
        // a lane past the end works on group 0 and keeps nothing
        const bool valid = k0 + tid < ngroups;
        const int rr = valid ? r : 0, w = valid ? wg * G : 0;
        const uint32_t* srow = x.s_src + (size_t)(x.HB + rr) * SW + (BLOCKS ? 4 : 0);
        uint32_t up[G], dn[G], sm[G], tg[G], hz[G];
        load_group<G>(srow + w - SW, up);
        load_group<G>(srow + w + SW, dn);
        load_group<G>(srow + w, sm);
        load_group<G>(x.s_tgt + (size_t)rr * CW + w, tg);
        if ((rr + x.par0) & 1) {
            const uint32_t next = srow[BLOCKS ? w + G : ((w + G == W) ? 0 : w + G)];
#pragma unroll
            for (int k = 0; k < G; ++k) hz[k] = __funnelshift_r(sm[k], k + 1 < G ? sm[k + 1] : next, 1);
        } else {
            const uint32_t prev = srow[BLOCKS ? w - 1 : ((w == 0) ? W - 1 : w - 1)];
#pragma unroll
            for (int k = 0; k < G; ++k) hz[k] = __funnelshift_l(k > 0 ? sm[k - 1] : prev, sm[k], 1);
        }
        const uint32_t pos0 = (uint32_t)(rr * W + w);  // from the tile's first word, in the plane
        const uint64_t q0 = x.q_tile + 8ull * pos0;  // the group's calls share q's high word
        uint32_t und[G], fm[G], sel[G], ql[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            uint32_t anti0;
            classify_word(tg[k], up[k], dn[k], sm[k], hz[k], all2, all4, zero2, zero4, fm[k], und[k], sel[k], anti0);
            if (!valid) und[k] = 0u;
            if (COUNT && valid) {
                ups += __popc(sm[k]);
                anti += anti0;
            }
            ql[k] = (uint32_t)q0 + 8u * k;
        }
        const uint32_t thr[2] = {t2, t4};
        // calls 0-1: nearly every warp needs both, so both are drawn without a vote
        bitsliced_below<G, 2, 0, 2, true, false>(und, fm, sel, sel, ql, group_consts(x, pc_tile, q0), x.key, thr);
        // the target words again, so that they need not stay in registers above
        uint32_t nw[G];
        if constexpr (G == 4) {
            const uint4 tq = ld_shared_v4(x.s_tgt + (size_t)rr * CW + w);
            nw[0] = tq.x ^ fm[0];
            nw[1] = tq.y ^ fm[1];
            nw[2] = tq.z ^ fm[2];
            nw[3] = tq.w ^ fm[3];
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) nw[k] = tg[k] ^ fm[k];
        }
        if constexpr (INPLACE) {
            uint32_t st[G];
#pragma unroll
            for (int k = 0; k < G; ++k) st[k] = und[k] != 0u ? nw[k] ^ fm[k] : nw[k];  // queued: the old word
            if (valid) store_group<G>(x.out + pos0, st);
        } else {
            if (valid) store_group<G>(x.out + pos0, nw);
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const bool pend = und[k] != 0u;
            if (COUNT && valid && !pend) {
                ups += __popc(nw[k]);
                anti += 4u * __popc(fm[k]) - 2u * __popc(fm[k] & sel[k]);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, pend);
            if (pend)
                wq[qn + __popc(bal & ((1u << lane) - 1u))] =
                    make_uint4(BLOCKS ? ((uint32_t)rr << 16) | (uint32_t)(w + k) : pos0 + k, und[k], fm[k], sel[k]);
            qn += __popc(bal);
            // the drain is inlined at few places: once per group (or per two words in
            // 512-thread CTAs, whose queues are shorter)
            constexpr int kEvery = (queue_cap(NT) - 31) / 32;
            if ((k + 1) % kEvery == 0 || k == G - 1) {
                if (qn >= 32) {
                    __syncwarp();  // pushes visible to the draining lanes
                    do {
                        drain_queue<COUNT, BLOCKS, TH>(x, pc_tile, wq, qn, 32, lane, ups, anti);
                    } while (qn >= 32);
                }
            }
        }
        r += step_r;
        wg += step_w;
        if (wg >= WG) {
            wg -= WG;
            ++r;
        }
    }
    if (qn > 0) {
        __syncwarp();
        drain_queue<COUNT, BLOCKS, TH>(x, pc_tile, wq, qn, qn, lane, ups, anti);
    }
}

// Register budgets: the single-lattice instance reads its descriptor from a
// __grid_constant__ parameter, so the key, thresholds and Philox constants sit in
// uniform registers and 2 CTAs of 256 fit at <= 128 registers; the general instance
// loads them per tile into ordinary registers and is allowed more (one CTA per
// 256 threads per SM), which is faster than spilling inside the random-number loop.
// TILES as for issue_tile: the single-lattice instance is compiled apart for whole rows
// (0) and for column blocks (1), and the multi-lattice instance for whole rows (0) and
// for either (2, once a lattice of the launch has column blocks), so that each carries
// only the tile code it needs.
template <int NT, bool ONE, int TILES, typename TH = RuntimeThresholds>
__global__ void __launch_bounds__(NT, (ONE ? (ISING_SWEEP_THREADS_PER_SM / NT > 0 ? ISING_SWEEP_THREADS_PER_SM / NT : 1)
                                           : (256 / NT > 0 ? 256 / NT : 1)))
    packed_half_sweep_kernel(TileTable tt, const __grid_constant__ LatticeDesc one, int colour, int step,
                             int* status, int stage_words_max, long long wait_limit, uint32_t extra_tx)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bars[0..1]: stage b filled (one arrival plus the copies' bytes); rel[b]: warps
    // done with the tile in stage b (the last one refills it); acc, done: the
    // single-lattice instance's block sums of the counts
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* rel = reinterpret_cast<uint32_t*>(smem_raw + 16);
    uint32_t* done = reinterpret_cast<uint32_t*>(smem_raw + 24);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw + 32);
    uint4* queues = reinterpret_cast<uint4*>(smem_raw + 128 + ((2 * (NT / 32) * 4 + 127) / 128) * 128);
    uint32_t* stages = reinterpret_cast<uint32_t*>(queues + (NT / 32) * queue_cap(NT));
    const int tid = threadIdx.x;
    const int count = ONE ? 1 : *tt.count;
    const int total = ONE ? (int)lattice_tiles(one.L, one.tile_rows, one.tile_words) : __ldg(tt.tile_start + count);

    // Stage b serves this CTA's tiles tn, tn + 2g, tn + 4g, ... (g = gridDim.x): fill it
    // with the first of them whose lattice is live (tiles of other lattices are skipped:
    // their iterations neither wait for the stage nor release it).
    auto fill = [&](int tn, int b) {
        for (; tn < total; tn += 2 * gridDim.x) {
            const TileInfo ti = tile_info<ONE>(tt, one, count, tn, step);
            if (!ti.live) continue;
            fence_proxy_async_smem();
            issue_tile<TILES>(desc_at<ONE>(tt, one, ti.lat), tn - tile_base<ONE>(tt, ti.lat), colour,
                       stages + (size_t)b * stage_words_max, &bars[b], extra_tx);
            return;
        }
    };

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        rel[0] = 0;
        rel[1] = 0;
        *done = 0;
        acc[0] = 0;
        acc[1] = 0;
        fence_mbarrier_init();
    }
    __syncthreads();  // the only CTA-wide barrier: from here on warps may run a tile apart
    if (tid == 0) {
        fill(blockIdx.x, 0);
        fill(blockIdx.x + gridDim.x, 1);
    }

    int buf = 0;
    uint32_t phase0 = 0, phase1 = 0;
    int t = blockIdx.x;

    int acc_lat = -1;          // lattice whose M/E counts are being accumulated
    uint32_t ups = 0, anti = 0;  // per-thread counts (colour-1 pass only)

    // warp reduction of (ups, anti); the warp's totals are counts of its own words, so
    // their 32-bit sums are exact.  The multi-lattice instance adds them to the lattice's
    // (M, E) slot per warp (warps reach a lattice change at different times); `last`
    // (the single-lattice instance after its last tile) sums the CTA's warps in shared
    // memory first, and the last warp to arrive adds the CTA's totals.
    auto flush = [&](int lat, bool last) {
        const uint32_t u = __reduce_add_sync(0xffffffffu, ups);
        const uint32_t a = __reduce_add_sync(0xffffffffu, anti);
        if ((tid & 31) == 0) {
            const LatticeDesc& d = desc_at<ONE>(tt, one, lat);
            int64_t* slot = d.hist + 2 * (int64_t)(d.sweep + (uint32_t)step);
            if (last) {
                atomicAdd(&acc[0], (unsigned long long)u);
                atomicAdd(&acc[1], (unsigned long long)a);
                __threadfence_block();
                if (atomicAdd(done, 1u) == NT / 32 - 1) {
                    __threadfence_block();
                    atomicAdd(reinterpret_cast<unsigned long long*>(slot), 2ull * atomicAdd(&acc[0], 0ull));
                    atomicAdd(reinterpret_cast<unsigned long long*>(slot + 1), 2ull * atomicAdd(&acc[1], 0ull));
                }
            } else {
                atomicAdd(reinterpret_cast<unsigned long long*>(slot), 2ull * u);
                atomicAdd(reinterpret_cast<unsigned long long*>(slot + 1), 2ull * a);
            }
        }
        ups = 0;
        anti = 0;
    };

    for (; t < total; t += gridDim.x) {
        const TileInfo cur = tile_info<ONE>(tt, one, count, t, step);
        if (cur.live) {
            const LatticeDesc& d = desc_at<ONE>(tt, one, cur.lat);
            const int local_tile = t - tile_base<ONE>(tt, cur.lat);
            const uint32_t parity = buf ? phase1 : phase0;
            bool ok = mbar_wait_bounded(&bars[buf], parity, wait_limit);
            if (buf)
                phase1 ^= 1;
            else
                phase0 ^= 1;
            // the warp decides together (a lane that left alone would break the warp's votes);
            // every wait of the CTA is bounded, so the other warps leave too
            if (!__all_sync(0xffffffffu, ok)) {
                atomicExch(status, kStatusTimeout);
                return;
            }
            if (colour == 1 && acc_lat != cur.lat) {
                if (acc_lat >= 0) flush(acc_lat, false);
                acc_lat = cur.lat;
            }
            const int W = d.W, L = d.L, TR = d.tile_rows, HB = d.halo_rows, CW = d.tile_words ? d.tile_words : W;
            const uint64_t key = d.key;
            const uint32_t sweep = d.sweep + (uint32_t)step;
            const uint32_t t2 = d.t2, t4 = d.t4, all2 = d.all2, all4 = d.all4;
            // row block and column block of the tile (a single column block of whole rows
            // when CW == W)
            const bool blocks = TILES == 1 || (TILES == 2 && CW != W);
            int i0 = local_tile * TR, w0 = 0;
            if (blocks) {
                const int ncb = W / CW;
                const int rb = local_tile / ncb, cb = local_tile - rb * ncb;
                i0 = rb * TR;
                w0 = cb * CW;
            }
            const int SW = blocks ? CW + 8 : W;
            uint32_t* out_plane = d.plane[colour];
            const uint32_t* s_src = stages + (size_t)buf * stage_words_max;
            const uint32_t* s_tgt = s_src + (size_t)(TR + 2 * HB) * SW;
            if (colour == 0 && local_tile == 0 && tid == 0) {
                // open this sweep's (M, E) slot: M = 2 * ups - N, E = 2 * anti - 2N
                int64_t* slot = d.hist + 2 * (int64_t)sweep;
                const int64_t N = (int64_t)L * L;
                slot[0] = -N;
                slot[1] = -2 * N;
            }
            // counter words q = i*L/8 + 8w stay below 2^32 when L <= 131072, so the
            // per-word Philox constants (which depend on q's high word) are fixed
            TileCtx x;
            x.s_src = s_src;
            x.s_tgt = s_tgt;
            x.out = out_plane + (size_t)i0 * W + w0;
            x.q_tile = 8ull * ((uint64_t)i0 * (uint64_t)W + (uint64_t)w0);
            x.key = key;
            x.sweep = sweep;
            x.t2 = t2;
            x.t4 = t4;
            x.all2 = all2;
            x.all4 = all4;
            x.zero2 = (t2 == 0u && all2 == 0u) ? ~0u : 0u;  // thresholds 0 (never accept) are
            x.zero4 = (t4 == 0u && all4 == 0u) ? ~0u : 0u;  // taken out of the test like 2^32
            x.W = W;
            x.HB = HB;
            x.colour = colour;
            x.CW = CW;
            x.SW = SW;
            x.par0 = (i0 + colour) & 1;
            x.q_small = L <= 131072;
            const PhiloxWordConsts pc_tile = philox_consts(key, 0u, sweep, (uint32_t)colour);
            uint4* wq = queues + (tid >> 5) * queue_cap(NT);
            const int nwords = TR * CW;
            if (colour == 1) {
                if (TILES != 0 && blocks)
                    update_tile<NT, 4, true, true, TH>(x, pc_tile, nwords, wq, ups, anti);
                else if (TILES == 1)
                    ;
                else if ((W & 3) == 0)
                    update_tile<NT, 4, true, false, TH>(x, pc_tile, nwords, wq, ups, anti);
                else if ((W & 1) == 0)
                    update_tile<NT, 2, true, false, TH>(x, pc_tile, nwords, wq, ups, anti);
                else
                    update_tile<NT, 1, true, false, TH>(x, pc_tile, nwords, wq, ups, anti);
            } else {
                if (TILES != 0 && blocks)
                    update_tile<NT, 4, false, true, TH>(x, pc_tile, nwords, wq, ups, anti);
                else if (TILES == 1)
                    ;
                else if ((W & 3) == 0)
                    update_tile<NT, 4, false, false, TH>(x, pc_tile, nwords, wq, ups, anti);
                else if ((W & 1) == 0)
                    update_tile<NT, 2, false, false, TH>(x, pc_tile, nwords, wq, ups, anti);
                else
                    update_tile<NT, 1, false, false, TH>(x, pc_tile, nwords, wq, ups, anti);
            }
            // this warp is done with the stage; the last warp to be done refills it
            __syncwarp();
            if ((tid & 31) == 0) {
                __threadfence_block();
                if (atomicAdd(&rel[buf], 1u) == NT / 32 - 1) {
                    rel[buf] = 0;
                    __threadfence_block();
                    fill(t + 2 * gridDim.x, buf);
                }
            }
        }
        buf ^= 1;
    }
    if (colour == 1 && acc_lat >= 0) flush(acc_lat, ONE);
}

}  // namespace sweep
}  // namespace ising

// Bit-packed checkerboard half-sweep (the paper's UpdateOptim, Algorithm 2, on
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
// plane by bit plane on whole words (word_update.cuh).
//
// Each persistent CTA walks the tile table: a tile is `tile_rows` full rows of
// one lattice.  Thread 0 stages the tile's source rows (plus the halo rows above
// and below, wrapped) and target rows into shared memory with bulk async copies
// (cp.async.bulk, completion on an mbarrier), double-buffered so the next tile
// lands while the current one is computed.
#include "ising_internal.cuh"
#include "philox.cuh"
#include "word_update.cuh"

// Threads per SM the register allocation must leave room for (a CTA of NT
// threads gets a register cap of 65536 / ISING_SWEEP_THREADS_PER_SM per thread).
#ifndef ISING_SWEEP_THREADS_PER_SM
#define ISING_SWEEP_THREADS_PER_SM 512
#endif

namespace ising {
namespace {


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

// Thread 0: stage the tile's rows.  Source rows [i0 - HB, i0 + TR + HB) (wrapped)
// and target rows [i0, i0 + TR).  Every copy starts on a 16-byte boundary: with
// W % 4 == 0 every row does (TR may then be 2); otherwise HB = 4 and tiles start
// on rows that are multiples of 4, so each copied block starts at a multiple of
// 4 rows.
__device__ __forceinline__ void issue_tile(const LatticeDesc& d, int local_tile, int colour, uint32_t* stage,
                                           uint64_t* bar, uint32_t extra_tx)
{
    const int W = d.W, L = d.L, TR = d.tile_rows, HB = d.halo_rows;
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

// Register budgets: the single-lattice instance reads its descriptor from a
// __grid_constant__ parameter, so the key, thresholds and Philox constants sit in
// uniform registers and 2 CTAs of 256 fit at <= 128 registers; the general instance
// loads them per tile into ordinary registers and is allowed more (one CTA per
// 256 threads per SM), which is faster than spilling inside the random-number loop.
template <int NT, bool ONE>
__global__ void __launch_bounds__(NT, (ONE ? (ISING_SWEEP_THREADS_PER_SM / NT > 0 ? ISING_SWEEP_THREADS_PER_SM / NT : 1)
                                           : (256 / NT > 0 ? 256 / NT : 1)))
    packed_half_sweep_kernel(TileTable tt, const __grid_constant__ LatticeDesc one, int colour, int step,
                             int* status, int stage_words_max, long long wait_limit, uint32_t extra_tx)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* red = reinterpret_cast<uint32_t*>(smem_raw + 16);  // 2 * NT/32 words
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem_raw + 128 + ((2 * (NT / 32) * 4 + 127) / 128) * 128);
    const int tid = threadIdx.x;
    const int count = ONE ? 1 : *tt.count;
    const int total = ONE ? one.L / one.tile_rows : __ldg(tt.tile_start + count);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbarrier_init();
    }
    __syncthreads();

    int buf = 0;
    uint32_t phase0 = 0, phase1 = 0;
    int t = blockIdx.x;
    TileInfo cur = {0, false};
    if (t < total) {
        cur = tile_info<ONE>(tt, one, count, t, step);
        if (cur.live && tid == 0)
            issue_tile(desc_at<ONE>(tt, one, cur.lat), t - tile_base<ONE>(tt, cur.lat), colour, stages, &bars[0],
                       extra_tx);
    }

    int acc_lat = -1;          // lattice whose M/E counts are being accumulated
    uint32_t ups = 0, anti = 0;  // per-thread counts (colour-1 pass only)

    auto flush = [&](int lat) {
        // block reduction of (ups, anti) then one pair of 64-bit atomics
        const uint32_t u = __reduce_add_sync(0xffffffffu, ups);
        const uint32_t a = __reduce_add_sync(0xffffffffu, anti);
        if ((tid & 31) == 0) {
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
            const LatticeDesc& d = desc_at<ONE>(tt, one, lat);
            int64_t* slot = d.hist + 2 * (int64_t)(d.sweep + (uint32_t)step);
            atomicAdd(reinterpret_cast<unsigned long long*>(slot), 2ull * su);
            atomicAdd(reinterpret_cast<unsigned long long*>(slot + 1), 2ull * sa);
        }
        __syncthreads();
        ups = 0;
        anti = 0;
    };

    for (; t < total; t += gridDim.x) {
        const int tn = t + gridDim.x;
        TileInfo nxt = {0, false};
        if (tn < total) {
            nxt = tile_info<ONE>(tt, one, count, tn, step);
            if (nxt.live && tid == 0) {
                fence_proxy_async_smem();
                issue_tile(desc_at<ONE>(tt, one, nxt.lat), tn - tile_base<ONE>(tt, nxt.lat), colour,
                           stages + (size_t)(buf ^ 1) * stage_words_max, &bars[buf ^ 1], extra_tx);
            }
        }
        if (cur.live) {
            const LatticeDesc& d = desc_at<ONE>(tt, one, cur.lat);
            const int local_tile = t - tile_base<ONE>(tt, cur.lat);
            const uint32_t parity = buf ? phase1 : phase0;
            bool ok = mbar_wait_bounded(&bars[buf], parity, wait_limit);
            if (buf)
                phase1 ^= 1;
            else
                phase0 ^= 1;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicExch(status, kStatusTimeout);
                // give copies still in flight a bounded chance to land before exiting
                if (nxt.live) mbar_wait_bounded(&bars[buf ^ 1], buf ? phase0 : phase1, wait_limit);
                return;
            }
            if (colour == 1 && acc_lat != cur.lat) {
                if (acc_lat >= 0) flush(acc_lat);
                acc_lat = cur.lat;
            }
            const int W = d.W, L = d.L, TR = d.tile_rows, HB = d.halo_rows;
            const uint64_t key = d.key;
            const uint32_t sweep = d.sweep + (uint32_t)step;
            const uint32_t t2 = d.t2, t4 = d.t4, all2 = d.all2, all4 = d.all4;
            const int i0 = local_tile * TR;
            uint32_t* out_plane = d.plane[colour];
            const uint32_t* s_src = stages + (size_t)buf * stage_words_max;
            const uint32_t* s_tgt = s_src + (size_t)(TR + 2 * HB) * W;
            if (colour == 0 && local_tile == 0 && tid == 0) {
                // open this sweep's (M, E) slot: M = 2 * ups - N, E = 2 * anti - 2N
                int64_t* slot = d.hist + 2 * (int64_t)sweep;
                const int64_t N = (int64_t)L * L;
                slot[0] = -N;
                slot[1] = -2 * N;
            }
            // counter words q = i*L/8 + 8w stay below 2^32 when L <= 131072, so the
            // per-word Philox constants (which depend on q's high word) are fixed
            const bool q_small = L <= 131072;
            const PhiloxWordConsts pc_tile = philox_consts(key, 0u, sweep, (uint32_t)colour);
            const int nwords = TR * W;
            // Four (or two) adjacent words per thread and iteration: one 128-bit (or
            // 64-bit) shared-memory load per neighbour row and one global store, and
            // one index step, per group of words.
            if ((W & 3) == 0) {
                const int W4 = W >> 2, nquads = nwords >> 2;
                const int step_r = NT / W4, step_w = NT - step_r * W4;
                int r = tid / W4, w4 = tid - r * W4;
                for (int idx4 = tid; idx4 < nquads; idx4 += NT) {
                    const int i = i0 + r;
                    const int w = 4 * w4;
                    const uint32_t* srow = s_src + (size_t)(HB + r) * W;
                    const uint4 upq = *reinterpret_cast<const uint4*>(srow + w - W);
                    const uint4 dnq = *reinterpret_cast<const uint4*>(srow + w + W);
                    const uint4 smq = *reinterpret_cast<const uint4*>(srow + w);
                    const uint4 tgq = *reinterpret_cast<const uint4*>(s_tgt + (size_t)r * W + w);
                    const int par = (i + colour) & 1;
                    uint32_t hz[4];
                    if (par) {
                        const uint32_t nextw = srow[(w + 4 == W) ? 0 : w + 4];
                        hz[0] = __funnelshift_r(smq.x, smq.y, 1);
                        hz[1] = __funnelshift_r(smq.y, smq.z, 1);
                        hz[2] = __funnelshift_r(smq.z, smq.w, 1);
                        hz[3] = __funnelshift_r(smq.w, nextw, 1);
                    } else {
                        const uint32_t prevw = srow[(w == 0) ? W - 1 : w - 1];
                        hz[0] = __funnelshift_l(prevw, smq.x, 1);
                        hz[1] = __funnelshift_l(smq.x, smq.y, 1);
                        hz[2] = __funnelshift_l(smq.y, smq.z, 1);
                        hz[3] = __funnelshift_l(smq.z, smq.w, 1);
                    }
                    const uint64_t q0 = (uint64_t)i * (uint64_t)(L >> 3) + 8ull * (uint64_t)w;
                    const PhiloxWordConsts pc =
                        q_small ? pc_tile : philox_consts(key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
                    const uint32_t up[4] = {upq.x, upq.y, upq.z, upq.w}, dn[4] = {dnq.x, dnq.y, dnq.z, dnq.w};
                    const uint32_t sm[4] = {smq.x, smq.y, smq.z, smq.w}, tg[4] = {tgq.x, tgq.y, tgq.z, tgq.w};
                    const uint32_t ql[4] = {(uint32_t)q0, (uint32_t)q0 + 8u, (uint32_t)q0 + 16u, (uint32_t)q0 + 24u};
                    // the random-number loop runs on two words at a time: a thread stops
                    // drawing once both are decided, and a warp once all its lanes are, so
                    // the smaller group draws fewer calls at warp level than all four
                    // words together would (the pair interleaves two calls)
                    uint32_t f[4];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint32_t a_t[2] = {tg[2 * hh], tg[2 * hh + 1]}, a_u[2] = {up[2 * hh], up[2 * hh + 1]};
                        const uint32_t a_d[2] = {dn[2 * hh], dn[2 * hh + 1]}, a_s[2] = {sm[2 * hh], sm[2 * hh + 1]};
                        const uint32_t a_h[2] = {hz[2 * hh], hz[2 * hh + 1]}, a_q[2] = {ql[2 * hh], ql[2 * hh + 1]};
                        uint32_t a_f[2];
                        if (colour == 1)
                            flip_masks<2, true>(a_t, a_u, a_d, a_s, a_h, a_q, pc, key, t2, t4, all2, all4, a_f, ups, anti);
                        else
                            flip_masks<2, false>(a_t, a_u, a_d, a_s, a_h, a_q, pc, key, t2, t4, all2, all4, a_f, ups, anti);
                        f[2 * hh] = a_f[0];
                        f[2 * hh + 1] = a_f[1];
                    }
                    // the target words again from shared memory, so that they need not
                    // stay in registers across the random-number loop
                    const uint4 tq = ld_shared_v4(s_tgt + (size_t)r * W + w);
                    const uint4 nq = make_uint4(tq.x ^ f[0], tq.y ^ f[1], tq.z ^ f[2], tq.w ^ f[3]);
                    *reinterpret_cast<uint4*>(out_plane + (size_t)i * W + w) = nq;
                    if (colour == 1) ups += __popc(nq.x) + __popc(nq.y) + __popc(nq.z) + __popc(nq.w);
                    r += step_r;
                    w4 += step_w;
                    if (w4 >= W4) {
                        w4 -= W4;
                        ++r;
                    }
                }
            } else if ((W & 1) == 0) {
                // pairs of adjacent words (W even but not a multiple of 4)
                const int W2 = W >> 1, npairs = nwords >> 1;
                const int step_r = NT / W2, step_w = NT - step_r * W2;
                int r = tid / W2, w2 = tid - r * W2;
                for (int idx2 = tid; idx2 < npairs; idx2 += NT) {
                    const int i = i0 + r;
                    const int w = 2 * w2;
                    const uint32_t* srow = s_src + (size_t)(HB + r) * W;
                    const uint2 upp = *reinterpret_cast<const uint2*>(srow + w - W);
                    const uint2 dnp = *reinterpret_cast<const uint2*>(srow + w + W);
                    const uint2 smp = *reinterpret_cast<const uint2*>(srow + w);
                    const uint2 tgp = *reinterpret_cast<const uint2*>(s_tgt + (size_t)r * W + w);
                    const int par = (i + colour) & 1;
                    uint32_t hz0, hz1;
                    if (par) {
                        const uint32_t nextw = srow[(w + 2 == W) ? 0 : w + 2];
                        hz0 = __funnelshift_r(smp.x, smp.y, 1);
                        hz1 = __funnelshift_r(smp.y, nextw, 1);
                    } else {
                        const uint32_t prevw = srow[(w == 0) ? W - 1 : w - 1];
                        hz0 = __funnelshift_l(prevw, smp.x, 1);
                        hz1 = __funnelshift_l(smp.x, smp.y, 1);
                    }
                    const uint64_t q0 = (uint64_t)i * (uint64_t)(L >> 3) + 8ull * (uint64_t)w;
                    const PhiloxWordConsts pc =
                        q_small ? pc_tile : philox_consts(key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
                    uint32_t f[2];
                    {
                        const uint32_t t2w[2] = {tgp.x, tgp.y};
                        const uint32_t u2[2] = {upp.x, upp.y}, d2[2] = {dnp.x, dnp.y}, m2[2] = {smp.x, smp.y};
                        const uint32_t z2[2] = {hz0, hz1}, ql[2] = {(uint32_t)q0, (uint32_t)q0 + 8u};
                        if (colour == 1)
                            flip_masks<2, true>(t2w, u2, d2, m2, z2, ql, pc, key, t2, t4, all2, all4, f, ups, anti);
                        else
                            flip_masks<2, false>(t2w, u2, d2, m2, z2, ql, pc, key, t2, t4, all2, all4, f, ups, anti);
                    }
                    const uint2 nw = make_uint2(tgp.x ^ f[0], tgp.y ^ f[1]);
                    *reinterpret_cast<uint2*>(out_plane + (size_t)i * W + w) = nw;
                    if (colour == 1) ups += __popc(nw.x) + __popc(nw.y);
                    r += step_r;
                    w2 += step_w;
                    if (w2 >= W2) {
                        w2 -= W2;
                        ++r;
                    }
                }
            } else {
            // (row, word) of idx = tid + k*NT, advanced without a division per word
            const int step_r = NT / W, step_w = NT - step_r * W;
            int r = tid / W, w = tid - r * W;
            for (int idx = tid; idx < nwords; idx += NT) {
                const int i = i0 + r;
                const uint32_t* srow = s_src + (size_t)(HB + r) * W;
                const uint32_t up = srow[w - W];
                const uint32_t down = srow[w + W];
                const uint32_t same = srow[w];
                const int par = (i + colour) & 1;
                uint32_t hz;
                if (par) {
                    const uint32_t nextw = srow[(w + 1 == W) ? 0 : w + 1];
                    hz = __funnelshift_r(same, nextw, 1);
                } else {
                    const uint32_t prevw = srow[(w == 0) ? W - 1 : w - 1];
                    hz = __funnelshift_l(prevw, same, 1);
                }
                const uint32_t tw = s_tgt[idx];
                const uint64_t q0 = (uint64_t)i * (uint64_t)(L >> 3) + 8ull * (uint64_t)w;
                const PhiloxWordConsts pc =
                    q_small ? pc_tile : philox_consts(key, (uint32_t)(q0 >> 32), sweep, (uint32_t)colour);
                uint32_t f[1];
                {
                    const uint32_t t1[1] = {tw};
                    const uint32_t u1[1] = {up}, d1[1] = {down}, m1[1] = {same}, z1[1] = {hz}, ql[1] = {(uint32_t)q0};
                    if (colour == 1)
                        flip_masks<1, true>(t1, u1, d1, m1, z1, ql, pc, key, t2, t4, all2, all4, f, ups, anti);
                    else
                        flip_masks<1, false>(t1, u1, d1, m1, z1, ql, pc, key, t2, t4, all2, all4, f, ups, anti);
                }
                out_plane[(size_t)i * W + w] = tw ^ f[0];
                if (colour == 1) ups += __popc(tw ^ f[0]);
                r += step_r;
                w += step_w;
                if (w >= W) {
                    w -= W;
                    ++r;
                }
            }
        }
            }
        __syncthreads();
        buf ^= 1;
        cur = nxt;
    }
    if (colour == 1 && acc_lat >= 0) flush(acc_lat);
}

// After `steps` sweeps: advance each live lattice's sweep counter (bounded by its target).
__global__ void packed_advance_kernel(LatticeDesc* desc, const int32_t* count, int steps)
{
    const int n = *count;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        LatticeDesc& d = desc[l];
        if (!d.active) continue;
        const uint64_t nxt = (uint64_t)d.sweep + (uint64_t)steps;
        d.sweep = (uint32_t)(nxt < d.target ? nxt : (uint64_t)(d.sweep < d.target ? d.target : d.sweep));
    }
}

}  // namespace

int packed_smem_header_bytes(int threads)
{
    return 128 + ((2 * (threads / 32) * 4 + 127) / 128) * 128;
}

template <int NT>
void launch_nt(const TileTable& tt, const LatticeDesc* one, int colour, int step, int* status, int grid, size_t smem,
               int stage_words, cudaStream_t s, long long wait_limit, uint32_t extra_tx)
{
    if (one)
        packed_half_sweep_kernel<NT, true><<<grid, NT, smem, s>>>(tt, *one, colour, step, status, stage_words,
                                                                  wait_limit, extra_tx);
    else
        packed_half_sweep_kernel<NT, false><<<grid, NT, smem, s>>>(tt, LatticeDesc{}, colour, step, status,
                                                                   stage_words, wait_limit, extra_tx);
}

cudaError_t launch_packed_half_sweep(const TileTable& tt, int colour, int step, int* status, int grid, int threads,
                                     int smem_stage_bytes, cudaStream_t s, long long wait_limit, uint32_t extra_tx,
                                     const LatticeDesc* one)
{
    const int stage_words = smem_stage_bytes / 4;
    const size_t smem = (size_t)packed_smem_header_bytes(threads) + 2 * (size_t)smem_stage_bytes;
    switch (threads) {
    case 128:
        launch_nt<128>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx);
        break;
    case 256:
        launch_nt<256>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx);
        break;
    case 512:
        launch_nt<512>(tt, one, colour, step, status, grid, smem, stage_words, s, wait_limit, extra_tx);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NT>
cudaError_t set_limit_nt(size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(packed_half_sweep_kernel<NT, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(packed_half_sweep_kernel<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

cudaError_t packed_set_smem_limit(int threads, size_t bytes)
{
    switch (threads) {
    case 128:
        return set_limit_nt<128>(bytes);
    case 256:
        return set_limit_nt<256>(bytes);
    case 512:
        return set_limit_nt<512>(bytes);
    default:
        return cudaErrorInvalidValue;
    }
}

template <int NT>
cudaError_t occupancy_nt(size_t smem, int* blocks_per_sm, bool one)
{
    return one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, packed_half_sweep_kernel<NT, true>, NT, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, packed_half_sweep_kernel<NT, false>, NT,
                                                               smem);
}

cudaError_t packed_occupancy(int threads, size_t smem, int* blocks_per_sm, bool one)
{
    switch (threads) {
    case 128:
        return occupancy_nt<128>(smem, blocks_per_sm, one);
    case 256:
        return occupancy_nt<256>(smem, blocks_per_sm, one);
    case 512:
        return occupancy_nt<512>(smem, blocks_per_sm, one);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_packed_advance(LatticeDesc* desc, const int32_t* count, int max_count, int steps, cudaStream_t s)
{
    const int threads = 128;
    const int grid = (max_count + threads - 1) / threads;
    packed_advance_kernel<<<grid > 0 ? grid : 1, threads, 0, s>>>(desc, count, steps);
    return cudaGetLastError();
}

}  // namespace ising

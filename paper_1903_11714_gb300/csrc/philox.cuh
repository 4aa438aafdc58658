// Device-side Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), specialised to the counter layout of the
// sweep: counter = (q low 32, q high 32, sweep, colour), key = (seed low, seed high).
//
// The draw replaces the paper's random_uniform (Algorithms 1-2): the uniform of a
// site of colour-plane index p is output word (p & 3) of the call with q = p >> 2.
//
// One Philox round maps (x0,x1,x2,x3) under round key (k0,k1) to
//   (hi(B*x2) ^ x1 ^ k0, lo(B*x2), hi(A*x0) ^ x3 ^ k1, lo(A*x0)),
// A = 0xD2511F53, B = 0xCD9E8D57; the key grows by (0x9E3779B9, 0xBB67AE85) per round.
//
// Within one 32-site word the eight calls differ only in counter word 0, so the
// products that involve only (q high, sweep, colour, key) are computed once per
// word: B*sweep in round 1 and A*x0 in round 2.  That removes 2 of the 20
// 32x32->64 multiplies per call without changing a single output bit.
#pragma once
#include <cstdint>

namespace ising {

constexpr uint32_t kPhiloxA = 0xD2511F53u;
constexpr uint32_t kPhiloxB = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;

__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t x, uint32_t& hi, uint32_t& lo)
{
    const uint64_t p = (uint64_t)a * (uint64_t)x;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Values shared by every call of one (key, counter-high, sweep, colour).
struct PhiloxWordConsts {
    uint32_t r1_x0, r1_x1;  // round-1 outputs 0 and 1 (independent of counter word 0)
    uint32_t r1_k;          // colour ^ k1 (xored into round-1 output 2)
    uint32_t r2_y0;         // round-1 output 1 ^ round-2 k0
    uint32_t r2_hi, r2_lo;  // hi / lo of A * r1_x0, with hi pre-xored by round-2 k1
};

__device__ __forceinline__ PhiloxWordConsts philox_consts(uint64_t key, uint32_t q_hi, uint32_t sweep,
                                                          uint32_t colour)
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    PhiloxWordConsts c;
    uint32_t hi, lo;
    mulhilo(kPhiloxB, sweep, hi, lo);
    c.r1_x0 = hi ^ q_hi ^ k0;
    c.r1_x1 = lo;
    c.r1_k = colour ^ k1;
    c.r2_y0 = lo ^ (k0 + kWeyl0);
    mulhilo(kPhiloxA, c.r1_x0, hi, lo);
    c.r2_hi = hi ^ (k1 + kWeyl1);
    c.r2_lo = lo;
    return c;
}

// Full ten rounds for counter word 0 = q_lo; writes the four output words.
__device__ __forceinline__ void philox_call(uint32_t q_lo, const PhiloxWordConsts& c, uint64_t key,
                                            uint32_t& o0, uint32_t& o1, uint32_t& o2, uint32_t& o3)
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    uint32_t hi, lo;
    // round 1: only the A * counter-word-0 product depends on the call
    mulhilo(kPhiloxA, q_lo, hi, lo);
    const uint32_t x2 = hi ^ c.r1_k;
    const uint32_t x3 = lo;
    // round 2: B * x2 depends on the call, A * x0 does not
    mulhilo(kPhiloxB, x2, hi, lo);
    uint32_t y0 = hi ^ c.r2_y0;
    uint32_t y1 = lo;
    uint32_t y2 = c.r2_hi ^ x3;
    uint32_t y3 = c.r2_lo;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t rk0 = k0 + (uint32_t)r * kWeyl0;
        const uint32_t rk1 = k1 + (uint32_t)r * kWeyl1;
        uint32_t h0, l0, h1, l1;
        mulhilo(kPhiloxA, y0, h0, l0);
        mulhilo(kPhiloxB, y2, h1, l1);
        const uint32_t n0 = h1 ^ y1 ^ rk0;
        const uint32_t n2 = h0 ^ y3 ^ rk1;
        y0 = n0;
        y1 = l1;
        y2 = n2;
        y3 = l0;
    }
    o0 = y0;
    o1 = y1;
    o2 = y2;
    o3 = y3;
}

// The eight calls of one 32-site word (counter word 0 = q_lo .. q_lo+7), advanced
// round by round together so the multiplies of different calls overlap, with
// each round key formed once per round for all eight.  out[4 j + m] is output
// word m of call j, i.e. the draw of the word's site 4 j + m.
__device__ __forceinline__ void philox_word8(uint32_t q_lo, const PhiloxWordConsts& c, uint64_t key,
                                             uint32_t out[32])
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    uint32_t y0[8], y1[8], y2[8], y3[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t hi, lo;
        mulhilo(kPhiloxA, q_lo + (uint32_t)j, hi, lo);  // round 1, counter-dependent half
        const uint32_t x2 = hi ^ c.r1_k;
        const uint32_t x3 = lo;
        mulhilo(kPhiloxB, x2, hi, lo);  // round 2, counter-dependent half
        y0[j] = hi ^ c.r2_y0;
        y1[j] = lo;
        y2[j] = c.r2_hi ^ x3;
        y3[j] = c.r2_lo;
    }
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t rk0 = k0 + (uint32_t)r * kWeyl0;
        const uint32_t rk1 = k1 + (uint32_t)r * kWeyl1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t h0, l0, h1, l1;
            mulhilo(kPhiloxA, y0[j], h0, l0);
            mulhilo(kPhiloxB, y2[j], h1, l1);
            const uint32_t n0 = h1 ^ y1[j] ^ rk0;
            const uint32_t n2 = h0 ^ y3[j] ^ rk1;
            y0[j] = n0;
            y1[j] = l1;
            y2[j] = n2;
            y3[j] = l0;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        out[4 * j + 0] = y0[j];
        out[4 * j + 1] = y1[j];
        out[4 * j + 2] = y2[j];
        out[4 * j + 3] = y3[j];
    }
}

// Plain ten-round Philox4x32-10 on an arbitrary counter (used by tests of the
// device generator and by the start-state kernels).
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                                              uint32_t out[4])
{
    uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mulhilo(kPhiloxA, c0, h0, l0);
        mulhilo(kPhiloxB, c2, h1, l1);
        const uint32_t n0 = h1 ^ c1 ^ k0;
        const uint32_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

}  // namespace ising

// Device-side Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), specialised to the counter layout of the
// sweep: counter = (sweep, q low 32, colour, q high 32), key = (seed low, seed high).
//
// The draw replaces the paper's random_uniform (Algorithms 1-2): the uniform of a
// site of colour-plane index p is output word (p & 3) of the call with q = p >> 2.
//
// One Philox round maps (x0,x1,x2,x3) under round key (k0,k1) to
//   (hi(B*x2) ^ x1 ^ k0, lo(B*x2), hi(A*x0) ^ x3 ^ k1, lo(A*x0)),
// A = 0xD2511F53, B = 0xCD9E8D57; the key grows by (0x9E3779B9, 0xBB67AE85) per round.
//
// The calls of one sweep and colour differ only in q, and q enters through counter
// word 1, which no round-1 product reads.  Following one varying input through the
// rounds: round 1's two products (A*sweep, B*colour) are fixed; round 2's B*x2 is
// fixed (x2 = hi(A*sweep) ^ q_hi ^ k1); round 3's A*x0 is fixed (x0 of round 3 is
// built from round 2's fixed B product).  So 4 of the 20 32x32->64 products of a call
// are formed once per (sweep, colour, q high) and 16 per call remain, without
// changing a single output bit.
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

// Values shared by every call of one (key, sweep, colour, q high).  Round r of
// ten (r = 0..9) uses key (k0 + r*W0, k1 + r*W1).
struct PhiloxWordConsts {
    uint32_t x0k;  // round 1: output 0 = q_lo ^ x0k, x0k = hi(B*colour) ^ k0
    uint32_t y2k;  // round 2: output 2 = hi(A*x0) ^ y2k, y2k = lo(A*sweep) ^ round-2 k1
    uint32_t z0k;  // round 3: output 0 = hi(B*y2) ^ z0k (round 2's fixed output 1 ^ round-3 k0)
    uint32_t z2k;  // round 3: output 2 = y3 ^ z2k (hi of the fixed A product ^ round-3 k1)
    uint32_t z3;   // round 3: output 3, lo of the fixed A product
};

__device__ __forceinline__ PhiloxWordConsts philox_consts(uint64_t key, uint32_t q_hi, uint32_t sweep,
                                                          uint32_t colour)
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    PhiloxWordConsts c;
    uint32_t pa_hi, pa_lo, pb_hi, pb_lo;
    // round 1 on (sweep, q_lo, colour, q_hi)
    mulhilo(kPhiloxA, sweep, pa_hi, pa_lo);
    mulhilo(kPhiloxB, colour, pb_hi, pb_lo);
    c.x0k = pb_hi ^ k0;
    const uint32_t x1 = pb_lo;
    const uint32_t x2 = pa_hi ^ q_hi ^ k1;
    const uint32_t x3 = pa_lo;
    // round 2: B*x2 is fixed
    c.y2k = x3 ^ (k1 + kWeyl1);
    mulhilo(kPhiloxB, x2, pb_hi, pb_lo);
    const uint32_t y0 = pb_hi ^ x1 ^ (k0 + kWeyl0);
    const uint32_t y1 = pb_lo;
    // round 3: A*y0 is fixed
    mulhilo(kPhiloxA, y0, pa_hi, pa_lo);
    c.z0k = y1 ^ (k0 + 2u * kWeyl0);
    c.z2k = pa_hi ^ (k1 + 2u * kWeyl1);
    c.z3 = pa_lo;
    return c;
}

// The eight calls of one 32-site word, q_lo .. q_lo + 7 with q_lo % 8 == 0 (a word
// starts at a multiple of 32 sites, so q_lo + j = q_lo ^ j), advanced round by
// round together so the multiplies of different calls overlap, with each round key
// formed once per round for all eight.  out[4 j + m] is output word m of call j,
// i.e. the draw of the word's site 4 j + m.
__device__ __forceinline__ void philox_word8(uint32_t q_lo, const PhiloxWordConsts& c, uint64_t key,
                                             uint32_t out[32])
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    const uint32_t base = q_lo ^ c.x0k;
    uint32_t y0[8], y1[8], y2[8], y3[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t hi, lo;
        mulhilo(kPhiloxA, base ^ (uint32_t)j, hi, lo);  // round 2, the varying product
        const uint32_t r2_y2 = hi ^ c.y2k;
        const uint32_t r2_y3 = lo;
        mulhilo(kPhiloxB, r2_y2, hi, lo);  // round 3, the varying product
        y0[j] = hi ^ c.z0k;
        y1[j] = lo;
        y2[j] = r2_y3 ^ c.z2k;
        y3[j] = c.z3;
    }
#pragma unroll
    for (int r = 3; r < 10; ++r) {
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

// The call of site-group q (= colour-plane index >> 2) in the sweep's counter layout
// (sweep, q low 32, colour, q high 32).
__device__ __forceinline__ void site_philox(uint64_t q, uint32_t sweep, uint32_t colour, uint64_t key,
                                            uint32_t out[4])
{
    philox4x32_10(sweep, (uint32_t)q, colour, (uint32_t)(q >> 32), key, out);
}

}  // namespace ising

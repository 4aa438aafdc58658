// Device-side Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), specialised to the counter layout of the
// sweep: counter = (sweep, q low 32, colour, q high 32), key = (seed low, seed high).
//
// The draw replaces the paper's random_uniform (Algorithms 1-2).  The colour-plane
// indices 32g .. 32g+31 form plane word g (one 32-bit word of a bit plane); the
// word's 32 random words R_0 .. R_31 are the outputs of the eight calls
// q = 8g .. 8g+7 (R_k = output k & 3 of call q = 8g + k/4), and the uniform of the
// site at bit b is U = sum_k bit_b(R_k) 2^(31-k).  So R_k is bit plane 31 - k of
// the 32 uniforms of the word: a word-parallel comparison U < T can read R_0, R_1,
// ... and stop as soon as every site is decided, leaving later calls undrawn.
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
#include "ising_device.cuh"

namespace ising {

constexpr uint32_t kPhiloxA = 0xD2511F53u;
constexpr uint32_t kPhiloxB = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;

// The 32x32->64 product of a round, as its high and low halves formed by two 32-bit
// multiplies: measured 2-3 % faster in every sweep kernel than one 64-bit product,
// whose single wide multiply kept one integer pipe busier than the others.
__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t x, uint32_t& hi, uint32_t& lo)
{
    hi = __umulhi(a, x);
    lo = a * x;
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

// Call c (0..7) of G plane words at once: word k's call is q = q_lo[k] + c with
// q_lo[k] % 8 == 0 (so q_lo + c = q_lo ^ c), passed as base[k] = q_lo[k] ^ x0k.
// The G calls advance round by round together so that their multiplies overlap,
// with each round key formed once per round.  o[k][m] = output word m of word k's
// call, i.e. the random word R_{4c+m} of that plane word.
template <int G>
__device__ __forceinline__ void philox_calls(const uint32_t base[G], uint32_t c, const PhiloxWordConsts& pc,
                                             uint64_t key, uint32_t o[G][4])
{
    const uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    uint32_t y0[G], y1[G], y2[G], y3[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        uint32_t hi, lo;
        mulhilo(kPhiloxA, base[k] ^ c, hi, lo);  // round 2, the varying product
        const uint32_t r2_y2 = hi ^ pc.y2k;
        const uint32_t r2_y3 = lo;
        mulhilo(kPhiloxB, r2_y2, hi, lo);  // round 3, the varying product
        y0[k] = hi ^ pc.z0k;
        y1[k] = lo;
        y2[k] = r2_y3 ^ pc.z2k;
        y3[k] = pc.z3;
    }
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint32_t rk0 = k0 + (uint32_t)r * kWeyl0;
        const uint32_t rk1 = k1 + (uint32_t)r * kWeyl1;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            uint32_t h0, l0, h1, l1;
            mulhilo(kPhiloxA, y0[k], h0, l0);
            mulhilo(kPhiloxB, y2[k], h1, l1);
            const uint32_t n0 = h1 ^ y1[k] ^ rk0;
            const uint32_t n2 = h0 ^ y3[k] ^ rk1;
            y0[k] = n0;
            y1[k] = l1;
            y2[k] = n2;
            y3[k] = l0;
        }
    }
#pragma unroll
    for (int k = 0; k < G; ++k) {
        o[k][0] = y0[k];
        o[k][1] = y1[k];
        o[k][2] = y2[k];
        o[k][3] = y3[k];
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

// Hot start of plane word g: a site is +1 iff its uniform drawn with sweep slot
// 0xFFFFFFFF is below 2^31, i.e. iff its bit of R_0 (the top bit plane) is 0; so
// the word of +1 bits is ~R_0, one call per word.
__device__ __forceinline__ uint32_t hot_start_word(uint64_t g, uint32_t colour, uint64_t key)
{
    const uint64_t q = 8 * g;
    uint32_t out[4];
    philox4x32_10(0xFFFFFFFFu, (uint32_t)q, colour, (uint32_t)(q >> 32), key, out);
    return ~out[0];
}

}  // namespace ising

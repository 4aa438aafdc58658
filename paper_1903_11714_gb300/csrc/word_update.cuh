// The Metropolis update of 32-site words of a target colour plane (paper Sec. 3.1
// acceptance rule on the bit-packed colour planes of Sec. 3.2), shared by the
// tiled sweep kernel, the single-CTA resident kernel, the int8 kernel and the
// three-dimensional sweep.
#pragma once
#include "ising_device.cuh"

#include "philox.cuh"

namespace ising {

// Bit-sliced test U < T_h for the sites of G plane words.  A site's uniform U has
// bit 31 - k in bit plane R_k of its word (see philox.cuh), so comparing U with
// its threshold from the top bit down decides the site at the first plane where
// the two bits differ: U < T there iff the threshold's bit is 1.  Per plane and
// word that is four logic operations for all 32 sites; planes are drawn four at a
// time (one Philox call) and drawing stops once no site is undecided -- a word alone
// needs about two of its eight calls (the tiled kernels draw calls 0-1 in step with
// the warp and finish the ~10 % of words with sites left from a queue), against
// eight calls for whole 32-bit uniforms.  The decisions are those of the full 32-bit
// comparison, bit for bit.
//
// und[k]: sites of word k still to test (updated); lt[k]: sites found below their
// threshold (ORed into).  NTH thresholds t[0..NTH-1] (values min(T, 2^32 - 1)); a
// site's threshold is t[0] where selA, else t[1] where selB (NTH = 3), else the
// last one.  Sites whose threshold is 0 or 2^32 must not be in und.
//
// Calls C0 .. C1-1 (planes 4*C0 .. 4*C1-1) are drawn; sites still in und after
// call 7 are not below (U equals T).  VOTE: stop when no site of the whole warp is
// undecided (every lane of the warp must be present), else when none of this
// thread's is.  CHECK = false draws every call without that test: for calls that
// nearly every warp needs, so that the calls and their comparisons form one block
// of straight-line code whose multiplies and logic operations can interleave.
template <int G, int NTH, int C0 = 0, int C1 = 8, bool VOTE = false, bool CHECK = true>
__device__ __forceinline__ void bitsliced_below(uint32_t und[G], uint32_t lt[G], const uint32_t selA[G],
                                                const uint32_t selB[G], const uint32_t q_lo[G],
                                                const PhiloxWordConsts& pc, uint64_t key, const uint32_t (&t)[NTH])
{
    uint32_t base[G];
#pragma unroll
    for (int k = 0; k < G; ++k) base[k] = q_lo[k] ^ pc.x0k;
#pragma unroll
    for (int c = C0; c < C1; ++c) {
        uint32_t any = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) any |= und[k];
        if (CHECK && (VOTE ? !__any_sync(0xffffffffu, any != 0u) : any == 0u)) break;
        uint32_t o[G][4];
        philox_calls<G>(base, (uint32_t)c, pc, key, o);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int bit = 31 - (4 * c + m);
            // the threshold's bit in this plane, as a mask per threshold
            uint32_t K[NTH];
#pragma unroll
            for (int h = 0; h < NTH; ++h) K[h] = 0u - ((t[h] >> bit) & 1u);
#pragma unroll
            for (int k = 0; k < G; ++k) {
                uint32_t tm;
                if constexpr (NTH == 2) {
                    tm = (selA[k] & K[0]) | (~selA[k] & K[1]);
                } else {
                    const uint32_t rest = (selB[k] & K[1]) | (~selB[k] & K[2]);
                    tm = (selA[k] & K[0]) | (~selA[k] & rest);
                }
                const uint32_t x = und[k] & (o[k][m] ^ tm);  // decided in this plane
                lt[k] |= x & tm;                              // ... below: U's bit 0, T's bit 1
                und[k] &= ~x;
            }
        }
    }
}

// Flip masks f[k] of G adjacent 32-site target words t[k] from their four
// neighbour words; q_lo[k] = 8 * (plane word index) of word k.  The caller applies
// them (t ^ f) -- from a fresh read of the target words if it wants them out of
// registers during the random-number loop.  With COUNT, adds the fused observables
// of the updated words except the set bits of the new target words, which the
// caller adds: ups += set bits of the `same` source words, anti += anti-aligned
// target-source bonds after the update.  The bond count comes from the adder bits,
// so the neighbour words need not stay live across the loop: a site with n
// anti-aligned neighbours keeps n if it stays and has 4 - n if it flips, and f
// contains every site with n >= 2 (b1 | b2), so the word's total is
// popc(b0) + 2 popc(b1) + 4 popc(b2) + sum over f of (4 - 2n)
//   = popc(b0) - 2 popc(b1) - 4 popc(b2) + 4 popc(f) - 2 popc(f & b0).
// (Unsigned wrap-around is harmless: each thread's total is non-negative.)
// The two-dimensional word classes of one target word t from its four neighbour
// words: f = sites that flip without a test (h <= 0, or a threshold of 2^32), und =
// sites to test against T2 (sel = 1, h = 2) or T4 (sel = 0, h = 4), zero2/zero4 =
// ~0u for a threshold of 0 (never accept).  anti0 = popc(b0) - 2 popc(b1) -
// 4 popc(b2), the update-independent part of the bond count (see flip_masks).
__device__ __forceinline__ void classify_word(uint32_t t, uint32_t up, uint32_t down, uint32_t same, uint32_t hz,
                                              uint32_t all2, uint32_t all4, uint32_t zero2, uint32_t zero4,
                                              uint32_t& f, uint32_t& und, uint32_t& sel, uint32_t& anti0)
{
    // anti-aligned neighbour bits and their 4-input sum n = 4*b2 + 2*b1 + b0
    const uint32_t au = t ^ up, ad = t ^ down, as = t ^ same, ah = t ^ hz;
    const uint32_t s0 = au ^ ad, c0 = au & ad;
    const uint32_t s1 = as ^ ah, c1 = as & ah;
    const uint32_t b0 = s0 ^ s1, cc = s0 & s1;
    const uint32_t b1 = c0 ^ c1 ^ cc;
    const uint32_t b2 = c0 & c1;
    // n >= 2 (h <= 0): always; n == 1 (h = 2): U < T2; n == 0 (h = 4): U < T4
    const uint32_t always = b1 | b2;
    const uint32_t h2 = b0 & ~always, h4 = ~b0 & ~always;
    f = always | (h2 & all2) | (h4 & all4);
    und = (h2 & ~(all2 | zero2)) | (h4 & ~(all4 | zero4));
    sel = b0;
    anti0 = __popc(b0) - 2u * __popc(b1) - 4u * __popc(b2);
}

template <int G, bool COUNT>
__device__ __forceinline__ void flip_masks(const uint32_t t[G], const uint32_t up[G], const uint32_t down[G],
                                           const uint32_t same[G], const uint32_t hz[G], const uint32_t q_lo[G],
                                           const PhiloxWordConsts& pc, uint64_t key, uint32_t t2, uint32_t t4,
                                           uint32_t all2, uint32_t all4, uint32_t f[G], uint32_t& ups, uint32_t& anti)
{
    // thresholds 0 (never accept) are taken out of the test like 2^32 (always)
    const uint32_t zero2 = (t2 == 0u && all2 == 0u) ? ~0u : 0u, zero4 = (t4 == 0u && all4 == 0u) ? ~0u : 0u;
    const uint32_t thr[2] = {t2, t4};
    uint32_t und[G], sel[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        uint32_t anti0;
        classify_word(t[k], up[k], down[k], same[k], hz[k], all2, all4, zero2, zero4, f[k], und[k], sel[k], anti0);
        if (COUNT) {
            ups += __popc(same[k]);
            anti += anti0;
        }
    }
    bitsliced_below<G, 2>(und, f, sel, sel, q_lo, pc, key, thr);
    if (COUNT) {
#pragma unroll
        for (int k = 0; k < G; ++k) anti += 4u * __popc(f[k]) - 2u * __popc(f[k] & sel[k]);
    }
}

}  // namespace ising

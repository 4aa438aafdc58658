// The update of one 32-site word of the target colour plane (paper Sec. 3.1
// acceptance rule on the bit-packed colour planes of Sec. 3.2), shared by the
// tiled sweep kernel and the single-CTA resident kernel.
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace ising {

// New value of one 32-site target word.
__device__ __forceinline__ uint32_t update_word(uint32_t t, uint32_t up, uint32_t down, uint32_t same,
                                                uint32_t hz, uint32_t q_lo, const PhiloxWordConsts& pc,
                                                uint64_t key, uint32_t t2, uint32_t t4, uint32_t all2,
                                                uint32_t all4)
{
    // anti-aligned neighbour bits and their 4-input sum n_anti = 4*b2 + 2*b1 + b0
    const uint32_t au = t ^ up, ad = t ^ down, as = t ^ same, ah = t ^ hz;
    const uint32_t s0 = au ^ ad, c0 = au & ad;
    const uint32_t s1 = as ^ ah, c1 = as & ah;
    const uint32_t b0 = s0 ^ s1, cc = s0 & s1;
    const uint32_t b1 = c0 ^ c1 ^ cc;
    const uint32_t b2 = c0 & c1;

    uint32_t x[32];
    philox_word8(q_lo, pc, key, x);
    // Threshold tests as carry chains: sub.cc sets the carry flag iff x >= t (no
    // borrow), and addc doubles the mask and adds that flag, so after 32 steps bit b
    // of g holds [x[b] >= t]; two instructions per compare, no predicate-to-bit
    // packing.  q = ~g is the mask of x < t.
    uint32_t g2 = 0, g4 = 0;
#pragma unroll
    for (int b = 31; b >= 0; --b) {
        asm("{\n\t.reg .u32 d;\n\tsub.cc.u32 d, %1, %2;\n\taddc.u32 %0, %0, %0;\n\t}" : "+r"(g2) : "r"(x[b]), "r"(t2));
        asm("{\n\t.reg .u32 d;\n\tsub.cc.u32 d, %1, %2;\n\taddc.u32 %0, %0, %0;\n\t}" : "+r"(g4) : "r"(x[b]), "r"(t4));
    }
    const uint32_t q2 = all2 | ~g2;
    const uint32_t q4 = all4 | ~g4;
    // n_anti >= 2 (h <= 0): always; n_anti == 1 (h = 2): x < T2; n_anti == 0 (h = 4):
    // x < T4.  T4 <= T2, so q4 is a subset of q2 and ORing q4 everywhere is exact.
    const uint32_t flip = b1 | b2 | (b0 & q2) | q4;
    return t ^ flip;
}

}  // namespace ising

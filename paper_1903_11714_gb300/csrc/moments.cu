// Exact moments of the per-sweep magnetisation and energy (Sec. 4.1: average
// magnetisation and the Binder parameter U4 = 1 - <m^4> / (3 <m^2>^2)).
//
// Over the samples s in [first, first + count) the kernel forms the exact
// integer sums S1 = sum |M| (64-bit), S2 = sum M^2 (128-bit), S4 = sum M^4
// (256-bit: |M| can reach 2^32 at L = 65,536), SE = sum E (signed 128-bit) and
// SE2 = sum E^2 (128-bit).  Integer addition is order-free, so any thread order
// gives the same sums; FP64 is used only once, on those exact sums:
//   <|m|> = S1 / (n N), <m^2> = S2 / (n N^2), <m^4> = S4 / (n N^4),
//   <e> = SE / (n N), <e^2> = SE2 / (n N^2), U4 = 1 - <m^4> / (3 <m^2>^2).
#include "ising_internal.cuh"

namespace ising {
namespace {

constexpr int kThreads = 256;
constexpr int kLimbs = 11;  // S1 | S2 (2) | S4 (4) | SE (2) | SE2 (2)

template <int N>
__device__ __forceinline__ void add_limbs(uint64_t* a, const uint64_t* b)
{
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const uint64_t s = a[k] + b[k];
        const uint64_t c1 = s < a[k];
        const uint64_t s2 = s + carry;
        const uint64_t c2 = s2 < s;
        a[k] = s2;
        carry = c1 | c2;
    }
}

__device__ double u128_to_double(const uint64_t* v)
{
    return (double)v[1] * 18446744073709551616.0 + (double)v[0];
}

__global__ void __launch_bounds__(kThreads) moments_kernel(const int64_t* hist, int64_t first, int64_t count,
                                                           int64_t N, double* out6, uint64_t* sums_out)
{
    __shared__ uint64_t sh[kLimbs][kThreads];
    uint64_t acc[kLimbs];
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) acc[k] = 0;
    for (int64_t s = threadIdx.x; s < count; s += kThreads) {
        const int64_t M = hist[2 * (first + s)];
        const int64_t E = hist[2 * (first + s) + 1];
        const uint64_t a = M < 0 ? (uint64_t)(-M) : (uint64_t)M;
        // S1
        acc[0] += a;
        // S2: a^2 as (lo, hi)
        const uint64_t lo = a * a, hi = __umul64hi(a, a);
        const uint64_t sq[2] = {lo, hi};
        add_limbs<2>(acc + 1, sq);
        // S4: (hi 2^64 + lo)^2 = lo^2 + 2 lo hi 2^64 + hi^2 2^128
        const uint64_t p_ll[4] = {lo * lo, __umul64hi(lo, lo), 0, 0};
        const uint64_t x0 = lo * hi, x1 = __umul64hi(lo, hi);
        const uint64_t p_lh[4] = {0, x0 << 1, (x1 << 1) | (x0 >> 63), x1 >> 63};
        const uint64_t p_hh[4] = {0, 0, hi * hi, __umul64hi(hi, hi)};
        add_limbs<4>(acc + 3, p_ll);
        add_limbs<4>(acc + 3, p_lh);
        add_limbs<4>(acc + 3, p_hh);
        // SE (two's complement 128-bit)
        const uint64_t se[2] = {(uint64_t)E, E < 0 ? ~0ull : 0ull};
        add_limbs<2>(acc + 7, se);
        // SE2
        const uint64_t ae = E < 0 ? (uint64_t)(-E) : (uint64_t)E;
        const uint64_t e2[2] = {ae * ae, __umul64hi(ae, ae)};
        add_limbs<2>(acc + 9, e2);
    }
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            uint64_t a[kLimbs], b[kLimbs];
            for (int k = 0; k < kLimbs; ++k) {
                a[k] = sh[k][threadIdx.x];
                b[k] = sh[k][threadIdx.x + stride];
            }
            a[0] += b[0];
            add_limbs<2>(a + 1, b + 1);
            add_limbs<4>(a + 3, b + 3);
            add_limbs<2>(a + 7, b + 7);
            add_limbs<2>(a + 9, b + 9);
            for (int k = 0; k < kLimbs; ++k) sh[k][threadIdx.x] = a[k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        uint64_t t[kLimbs];
        for (int k = 0; k < kLimbs; ++k) {
            t[k] = sh[k][0];
            if (sums_out) sums_out[k] = t[k];
        }
        const double n = (double)count, dN = (double)N;
        const double s1 = (double)t[0];
        const double s2 = u128_to_double(t + 1);
        const double s4 = ((((double)t[6] * 18446744073709551616.0) + (double)t[5]) * 18446744073709551616.0 +
                           (double)t[4]) * 18446744073709551616.0 + (double)t[3];
        double se;
        if (t[8] >> 63) {  // negative: negate the 128-bit value
            const uint64_t nlo = ~t[7] + 1ull;
            const uint64_t nhi = ~t[8] + (nlo == 0 ? 1ull : 0ull);
            const uint64_t v[2] = {nlo, nhi};
            se = -u128_to_double(v);
        } else {
            se = u128_to_double(t + 7);
        }
        const double se2 = u128_to_double(t + 9);
        const double abs_m = s1 / (n * dN);
        const double m2 = s2 / (n * (dN * dN));
        const double m4 = s4 / (n * ((dN * dN) * (dN * dN)));
        out6[0] = abs_m;
        out6[1] = m2;
        out6[2] = m4;
        out6[3] = se / (n * dN);
        out6[4] = se2 / (n * (dN * dN));
        out6[5] = m2 > 0.0 ? 1.0 - m4 / (3.0 * m2 * m2) : 0.0;
    }
}

}  // namespace

cudaError_t launch_moments(const int64_t* hist, int64_t first, int64_t count, int64_t N, double* out6,
                           uint64_t* sums, cudaStream_t s)
{
    moments_kernel<<<1, kThreads, 0, s>>>(hist, first, count, N, out6, sums);
    return cudaGetLastError();
}

}  // namespace ising

/*
 * ising_oracle.c -- plain CPU oracle for the checkerboard Metropolis sweep of the
 * 2D nearest-neighbour Ising model on an L x L torus.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper: Sec. 3, Sec. 3.1 and Algorithms 1-2):
 *   H(sigma) = -J sum_<ij> sigma_i sigma_j - mu sum_i sigma_i with mu = 0, J = 1 on a
 *   torus (Sec. 3).  The lattice is coloured like a checkerboard; colour
 *   c(i,j) = (i+j) mod 2, 0 = black (the compact sub-lattices sigma_00 and sigma_11
 *   of Sec. 3.2), 1 = white.  One sweep updates every black site with the white
 *   sites fixed, then every white site with the black sites fixed (Sec. 3.1, the
 *   factorised transition kernel).  A site with h = sigma * nn (nn = sum of the four
 *   neighbours) is flipped with probability min{1, exp(-2 beta h)} (Sec. 3.1,
 *   acceptance rule with sigma* = -sigma; Algorithm 1's acceptance ratio with beta
 *   restored).
 *
 * Readings where the paper leaves the choice open (all stated in the design notes):
 *   - The uniform draw is a 32-bit word x from Philox4x32-10 (Salmon, Moraes,
 *     Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11); the
 *     test u < p with u = x / 2^32 becomes x < T_h, T_h = min(2^32, ceil(p 2^32)),
 *     p = exp(-2 beta h) evaluated in FP64 by the host libm.  h <= 0 always flips.
 *   - Site (i,j) of colour c has colour-plane index p = i*(L/2) + (j>>1); the
 *     plane indices 32g .. 32g+31 form plane word g = p >> 5, and b = p & 31 is
 *     the site's bit position in it.  Word g draws 32 random words R_0 .. R_31 per
 *     sweep: R_k is output word (k & 3) of Philox with key = (seed low 32, seed
 *     high 32) and counter = (sweep, q low 32, c, q high 32), q = 8g + (k >> 2).
 *     The site's uniform is U = sum_k bit_b(R_k) 2^(31-k): R_0 holds the top bit
 *     of the uniforms of all 32 sites of the word, R_31 the bottom bit.  (Every
 *     bit of U is an independent fair bit, as with a whole 32-bit draw; this
 *     assignment lets a word-parallel comparison stop at the first bits that
 *     decide it.)
 *   - Hot start: sigma = +1 iff the uniform drawn with sweep = 0xFFFFFFFF is
 *     below 2^31.  Cold start: all +1.
 *   - M = sum sigma; E = -sum_{i,j} sigma[i][j] (sigma[i+1][j] + sigma[i][j+1]),
 *     i.e. H with mu = 0, J = 1 over the 2N torus bonds.
 *
 * Pins (tests/test_oracle_*.py): Philox against cuRAND's host generator (key and
 * counter words 0-2) and its device API (word 3, on a GPU); thresholds against
 * 50-digit arithmetic; the chain against exact enumeration (4x4), the transfer
 * matrix (6x6, 8x8), Kaufman's finite-torus energy, Onsager's spontaneous
 * magnetisation; deterministic limits (beta = 0, zero temperature); the
 * incremental-energy invariant; exact stationarity of the quantised kernel.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11).  One round maps counter (c0,c1,c2,c3)
 * with round key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * with M0 = 0xD2511F53 and M1 = 0xCD9E8D57; between rounds the key is bumped by
 * the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.
 * ------------------------------------------------------------------------- */
ORACLE_API void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------------------
 * Acceptance thresholds.  T[0] is for h = 2 (p = exp(-4 beta)), T[1] for h = 4
 * (p = exp(-8 beta)).  p * 2^32 is exact in FP64 (a power-of-two scaling), so
 * the only rounding is the libm exp.  T = 2^32 means "always", T = 0 "never".
 * ------------------------------------------------------------------------- */
ORACLE_API void oracle_thresholds(double beta, uint64_t T[2])
{
    for (int n = 0; n < 2; ++n) {
        int h = 2 * (n + 1);
        double p = exp(-2.0 * beta * (double)h);
        double t = ceil(p * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        if (t < 0.0) t = 0.0;
        T[n] = (uint64_t)t;
    }
}

/* The Metropolis decision for one site: flip iff h <= 0, or the uniform word is
 * below the threshold of its h (Sec. 3.1). */
ORACLE_API int oracle_accept(int h, uint32_t x, uint64_t T2, uint64_t T4)
{
    if (h <= 0) return 1;
    if (h == 2) return (uint64_t)x < T2;
    return (uint64_t)x < T4; /* h == 4 */
}

static inline int64_t wrap(int64_t a, int64_t L)
{
    a %= L;
    return a < 0 ? a + L : a;
}

/* The 32 random words R_0 .. R_31 of plane word g for one sweep and colour (see header). */
ORACLE_API void oracle_word_randoms(uint64_t g, uint64_t seed, uint32_t sweep, int c, uint32_t R[32])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int n = 0; n < 8; ++n) {
        uint64_t q = 8 * g + (uint64_t)n;
        uint32_t ctr[4] = {sweep, (uint32_t)q, (uint32_t)c, (uint32_t)(q >> 32)};
        oracle_philox4x32_10(ctr, key, R + 4 * n);
    }
}

/* U of bit position b: bit b of R_k is the bit of weight 2^(31-k). */
static uint32_t uniform_of(const uint32_t R[32], int b)
{
    uint32_t u = 0;
    for (int k = 0; k < 32; ++k) u |= ((R[k] >> b) & 1u) << (31 - k);
    return u;
}

/* Uniforms of one row, colour c only, through a cache of the current plane word's
 * random words (a row of colour c holds whole plane words when L % 64 == 0 and
 * parts of two otherwise; the cache follows g either way). */
struct word_cache {
    uint64_t g;
    uint32_t R[32];
};

static uint32_t cached_uniform(struct word_cache *wc, uint64_t p, uint64_t seed, uint32_t sweep, int c)
{
    uint64_t g = p >> 5;
    if (g != wc->g) {
        oracle_word_randoms(g, seed, sweep, c, wc->R);
        wc->g = g;
    }
    return uniform_of(wc->R, (int)(p & 31));
}

/* Uniform of site (i,j) of colour c for the given sweep (see header). */
static uint32_t site_word(int64_t L, int64_t i, int64_t j, uint64_t seed, uint32_t sweep, int c)
{
    uint64_t p = (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(j >> 1);
    uint32_t R[32];
    oracle_word_randoms(p >> 5, seed, sweep, c, R);
    return uniform_of(R, (int)(p & 31));
}

ORACLE_API uint32_t oracle_site_word(int64_t L, int64_t i, int64_t j, uint64_t seed, uint32_t sweep, int c)
{
    return site_word(L, i, j, seed, sweep, c);
}

/* start: 0 = hot (iid +-1 from Philox, sweep slot 0xFFFFFFFF), 1 = cold (all +1). */
ORACLE_API void oracle_init(int8_t *s, int64_t L, uint64_t seed, int start)
{
#pragma omp parallel for schedule(static) if (L >= 64)
    for (int64_t i = 0; i < L; ++i) {
        struct word_cache wc[2] = {{UINT64_MAX, {0}}, {UINT64_MAX, {0}}};
        for (int64_t j = 0; j < L; ++j) {
            if (start == 1) {
                s[i * L + j] = 1;
            } else {
                int c = (int)((i + j) & 1);
                uint64_t p = (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(j >> 1);
                uint32_t x = cached_uniform(&wc[c], p, seed, 0xFFFFFFFFu, c);
                s[i * L + j] = (x < 0x80000000u) ? 1 : -1;
            }
        }
    }
}

/* M = sum sigma, E = -sum over the 2N torus bonds (H of Sec. 3, mu = 0, J = 1). */
ORACLE_API void oracle_observe(const int8_t *s, int64_t L, int64_t *M, int64_t *E)
{
    int64_t m = 0, e = 0;
#pragma omp parallel for reduction(+ : m, e) schedule(static) if (L >= 64)
    for (int64_t i = 0; i < L; ++i)
        for (int64_t j = 0; j < L; ++j) {
            int64_t v = s[i * L + j];
            m += v;
            e -= v * (s[wrap(i + 1, L) * L + j] + s[i * L + wrap(j + 1, L)]);
        }
    *M = m;
    *E = e;
}

/* One half-sweep of colour c (Algorithm 1's semantics, restricted to colour c as
 * in Algorithm 2).  words == NULL draws from Philox; otherwise words[i*L+j] is the
 * uniform word used at site (i,j) (a test hook for deterministic cases).
 * Returns the energy change sum of 2h over accepted flips. */
static int64_t half_sweep(int8_t *s, int64_t L, int c, uint64_t T2, uint64_t T4,
                          uint64_t seed, uint32_t sweep, const uint32_t *words)
{
    int64_t dE = 0;
#pragma omp parallel for reduction(+ : dE) schedule(static) if (L >= 64)
    for (int64_t i = 0; i < L; ++i) {
        /* The 32 same-colour sites of a plane word share its 32 random words; cache them. */
        struct word_cache wc = {UINT64_MAX, {0}};
        for (int64_t j = 0; j < L; ++j) {
            if (((i + j) & 1) != c) continue;
            int nn = s[wrap(i - 1, L) * L + j] + s[wrap(i + 1, L) * L + j]
                   + s[i * L + wrap(j - 1, L)] + s[i * L + wrap(j + 1, L)];
            int h = s[i * L + j] * nn;
            uint32_t x;
            if (words) {
                x = words[i * L + j];
            } else {
                uint64_t p = (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(j >> 1);
                x = cached_uniform(&wc, p, seed, sweep, c);
            }
            if (oracle_accept(h, x, T2, T4)) {
                s[i * L + j] = (int8_t)(-s[i * L + j]);
                dE += 2 * h;
            }
        }
    }
    return dE;
}

ORACLE_API int64_t oracle_half_sweep_words(int8_t *s, int64_t L, int c, uint64_t T2, uint64_t T4,
                                           const uint32_t *words)
{
    return half_sweep(s, L, c, T2, T4, 0, 0, words);
}

/* Runs sweeps sweep0 .. sweep0+nsweeps-1 (black then white each) on s.  Records
 * M[k], E[k] after each sweep when the arrays are non-NULL.  With check != 0
 * the energy is also carried incrementally (E += 2h per accepted flip) and
 * compared with the recomputed value after every half-sweep; returns the number
 * of mismatches (0 when the invariant holds). */
ORACLE_API int64_t oracle_run(int8_t *s, int64_t L, double beta, uint64_t seed, int64_t sweep0,
                              int64_t nsweeps, int64_t *M, int64_t *E, int check)
{
    uint64_t T[2];
    oracle_thresholds(beta, T);
    int64_t mism = 0, m0 = 0, e_inc = 0;
    if (check) oracle_observe(s, L, &m0, &e_inc);
    for (int64_t k = 0; k < nsweeps; ++k) {
        uint32_t sweep = (uint32_t)(sweep0 + k);
        for (int c = 0; c < 2; ++c) {
            int64_t dE = half_sweep(s, L, c, T[0], T[1], seed, sweep, NULL);
            if (check) {
                int64_t m, e;
                e_inc += dE;
                oracle_observe(s, L, &m, &e);
                if (e != e_inc) ++mism;
            }
        }
        if (M || E) {
            int64_t m, e;
            oracle_observe(s, L, &m, &e);
            if (M) M[k] = m;
            if (E) E[k] = e;
        }
    }
    return mism;
}

/* Light-cone evaluation of an h x w window of the lattice after nsweeps sweeps
 * from the start state, without simulating the whole torus.  A site's value
 * after t half-sweeps depends only on sites within Manhattan distance t, so a
 * buffer with a margin of R = 2*nsweeps cells on each side, updated on a region
 * that shrinks by one cell per half-sweep, reproduces the exact chain inside the
 * window.  Sites are addressed by global torus coordinates (i0+a) mod L,
 * (j0+b) mod L, so the random words and colours are those of the full run.
 * Returns 0, or -1 when the buffer cannot be allocated. */
ORACLE_API int oracle_window(int64_t L, double beta, uint64_t seed, int start, int64_t sweep0,
                             int64_t nsweeps, int64_t i0, int64_t j0, int64_t h, int64_t w,
                             int8_t *out)
{
    uint64_t T[2];
    oracle_thresholds(beta, T);
    int64_t R = 2 * nsweeps;
    int64_t H = h + 2 * R, W = w + 2 * R;
    int8_t *buf = (int8_t *)malloc((size_t)(H * W));
    if (!buf) return -1;
    /* Start state at global coordinates. */
#pragma omp parallel for schedule(static) if (L >= 64)
    for (int64_t a = 0; a < H; ++a) {
        struct word_cache wc[2] = {{UINT64_MAX, {0}}, {UINT64_MAX, {0}}};
        for (int64_t b = 0; b < W; ++b) {
            int64_t gi = wrap(i0 - R + a, L), gj = wrap(j0 - R + b, L);
            if (start == 1) {
                buf[a * W + b] = 1;
            } else {
                int cc = (int)((gi + gj) & 1);
                uint64_t p = (uint64_t)gi * (uint64_t)(L / 2) + (uint64_t)(gj >> 1);
                uint32_t x = cached_uniform(&wc[cc], p, seed, 0xFFFFFFFFu, cc);
                buf[a * W + b] = (x < 0x80000000u) ? 1 : -1;
            }
        }
    }
    for (int64_t t = 0; t < 2 * nsweeps; ++t) {
        uint32_t sweep = (uint32_t)(sweep0 + t / 2);
        int c = (int)(t & 1);
        int64_t lo = t + 1, hi_a = H - t - 1, hi_b = W - t - 1;
#pragma omp parallel for schedule(static) if (L >= 64)
        for (int64_t a = lo; a < hi_a; ++a) {
            struct word_cache wc = {UINT64_MAX, {0}};
            for (int64_t b = lo; b < hi_b; ++b) {
                int64_t gi = wrap(i0 - R + a, L), gj = wrap(j0 - R + b, L);
                if (((gi + gj) & 1) != c) continue;
                int nn = buf[(a - 1) * W + b] + buf[(a + 1) * W + b] + buf[a * W + b - 1] + buf[a * W + b + 1];
                int hh = buf[a * W + b] * nn;
                uint64_t p = (uint64_t)gi * (uint64_t)(L / 2) + (uint64_t)(gj >> 1);
                uint32_t x = cached_uniform(&wc, p, seed, sweep, c);
                if (oracle_accept(hh, x, T[0], T[1])) buf[a * W + b] = (int8_t)(-buf[a * W + b]);
            }
        }
    }
    for (int64_t a = 0; a < h; ++a)
        memcpy(out + a * w, buf + (a + R) * W + R, (size_t)w);
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Row-band forms, used only to time a bounded sample of a large lattice on the
 * host (the CPU baseline): the start state and the half-sweep of rows
 * [row0, row0 + nrows) of the full L x L lattice, with the same per-site rule,
 * keying and Philox as above.  The neighbour rows row0 - 1 and row0 + nrows are
 * read from s and must have been initialised by the caller.
 * ------------------------------------------------------------------------- */
ORACLE_API void oracle_init_rows(int8_t *s, int64_t L, uint64_t seed, int start, int64_t row0, int64_t nrows)
{
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nrows; ++a) {
        int64_t i = wrap(row0 + a, L);
        struct word_cache wc[2] = {{UINT64_MAX, {0}}, {UINT64_MAX, {0}}};
        for (int64_t j = 0; j < L; ++j) {
            if (start == 1) {
                s[i * L + j] = 1;
            } else {
                int c = (int)((i + j) & 1);
                uint64_t p = (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(j >> 1);
                uint32_t x = cached_uniform(&wc[c], p, seed, 0xFFFFFFFFu, c);
                s[i * L + j] = (x < 0x80000000u) ? 1 : -1;
            }
        }
    }
}

ORACLE_API int64_t oracle_half_sweep_rows(int8_t *s, int64_t L, int c, double beta, uint64_t seed, uint32_t sweep,
                                          int64_t row0, int64_t nrows)
{
    uint64_t T[2];
    oracle_thresholds(beta, T);
    int64_t dE = 0;
#pragma omp parallel for reduction(+ : dE) schedule(static)
    for (int64_t a = 0; a < nrows; ++a) {
        int64_t i = wrap(row0 + a, L);
        struct word_cache wc = {UINT64_MAX, {0}};
        for (int64_t j = 0; j < L; ++j) {
            if (((i + j) & 1) != c) continue;
            int nn = s[wrap(i - 1, L) * L + j] + s[wrap(i + 1, L) * L + j]
                   + s[i * L + wrap(j - 1, L)] + s[i * L + wrap(j + 1, L)];
            int h = s[i * L + j] * nn;
            uint64_t p = (uint64_t)i * (uint64_t)(L / 2) + (uint64_t)(j >> 1);
            if (oracle_accept(h, cached_uniform(&wc, p, seed, sweep, c), T[0], T[1])) {
                s[i * L + j] = (int8_t)(-s[i * L + j]);
                dE += 2 * h;
            }
        }
    }
    return dE;
}

/*
 * ising3d_oracle.c -- plain CPU oracle for the checkerboard Metropolis sweep of the
 * 3D nearest-neighbour Ising model on an X x Y x Z torus.
 *
 * TEST INFRASTRUCTURE ONLY, like ising_oracle.c (built into the same shared
 * object): only the tests, the package smoke check and the benchmark's CPU
 * baseline leg use it, and it shares no code, header or table with the CUDA path.
 *
 * What it computes: the Hamiltonian of Sec. 3 on the d-dimensional hypercubic
 * lattice, here d = 3, mu = 0, J = 1: H = -sum over nearest-neighbour pairs of
 * sigma_i sigma_j on the torus, i.e. the 3N bonds (s, s + e_x), (s, s + e_y),
 * (s, s + e_z).  The paper states that its checkerboard algorithm generalises to
 * three dimensions (Conclusion); the generalisation used here keeps every rule of
 * the 2D chain (Sec. 3.1 and Algorithms 1-2) and changes only the neighbourhood:
 *   - colour c(i,j,k) = (i+j+k) mod 2, black (0) then white (1) in every sweep;
 *     all six neighbours of a site have the other colour, so one half-sweep
 *     updates a colour with the other fixed (the factorised kernel of Sec. 3.1);
 *   - nn = sum of the six neighbours, h = sigma * nn in {-6, ..., 6}; the site
 *     flips with probability min{1, exp(-2 beta h)}: always for h <= 0, else iff
 *     the uniform word x is below T_h = min(2^32, ceil(exp(-2 beta h) 2^32)),
 *     h = 2, 4, 6, evaluated in FP64 by the host libm.
 *
 * Readings (the paper gives no 3D algorithm; these mirror the 2D readings):
 *   - Site (i,j,k) has colour-plane index p = (i*Y + j)*(Z/2) + (k>>1): the 2D
 *     index with the row (i,j) numbered i*Y + j.  Its uniform is drawn from p as
 *     in 2D: U = sum_k bit_{p & 31}(R_k) 2^(31-k) with R_0 .. R_31 the random words
 *     of plane word p >> 5 (oracle_word_randoms of ising_oracle.c).
 *   - Hot start: sigma = +1 iff the uniform drawn with sweep = 0xFFFFFFFF is below
 *     2^31; cold start all +1.
 *   - M = sum sigma; E = H = -sum over the 3N bonds.  A dimension of extent 2
 *     makes the two neighbours along it the same site, counted twice in nn and
 *     bonded twice in H, so the chain stays the Metropolis chain of that H.
 *   - All extents are even (so that the colouring is consistent on the torus).
 *
 * Pins (tests/test_oracle_3d.py): thresholds against 50-digit arithmetic; the
 * chain against exact enumeration on the 2x2x4 torus; exact stationarity of the
 * quantised half-sweep kernel; deterministic limits (beta = 0, zero temperature)
 * against a separately written numpy rule; the incremental-energy invariant.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_API __attribute__((visibility("default")))

/* The random words of one plane word, from ising_oracle.c (same shared object). */
void oracle_word_randoms(uint64_t g, uint64_t seed, uint32_t sweep, int c, uint32_t R[32]);

static inline int64_t wrap3(int64_t a, int64_t n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

/* Thresholds for h = 2, 4, 6: T[n] = min(2^32, ceil(exp(-2 beta h) 2^32)), h = 2(n+1). */
ORACLE_API void oracle3d_thresholds(double beta, uint64_t T[3])
{
    for (int n = 0; n < 3; ++n) {
        int h = 2 * (n + 1);
        double t = ceil(exp(-2.0 * beta * (double)h) * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        if (t < 0.0) t = 0.0;
        T[n] = (uint64_t)t;
    }
}

/* Metropolis decision of one site: flip iff h <= 0, or x below the threshold of h. */
ORACLE_API int oracle3d_accept(int h, uint32_t x, const uint64_t T[3])
{
    if (h <= 0) return 1;
    return (uint64_t)x < T[h / 2 - 1];
}

static uint32_t uniform3_of(const uint32_t R[32], int b)
{
    uint32_t u = 0;
    for (int k = 0; k < 32; ++k) u |= ((R[k] >> b) & 1u) << (31 - k);
    return u;
}

struct word_cache3 {
    uint64_t g;
    uint32_t R[32];
};

static uint32_t cached_uniform3(struct word_cache3 *wc, uint64_t p, uint64_t seed, uint32_t sweep, int c)
{
    if ((p >> 5) != wc->g) {
        wc->g = p >> 5;
        oracle_word_randoms(wc->g, seed, sweep, c, wc->R);
    }
    return uniform3_of(wc->R, (int)(p & 31));
}

static uint64_t plane_index3(int64_t Y, int64_t Z, int64_t i, int64_t j, int64_t k)
{
    return ((uint64_t)i * (uint64_t)Y + (uint64_t)j) * (uint64_t)(Z / 2) + (uint64_t)(k >> 1);
}

ORACLE_API uint32_t oracle3d_site_word(int64_t X, int64_t Y, int64_t Z, int64_t i, int64_t j, int64_t k,
                                       uint64_t seed, uint32_t sweep, int c)
{
    (void)X;
    struct word_cache3 wc = {UINT64_MAX, {0}};
    return cached_uniform3(&wc, plane_index3(Y, Z, i, j, k), seed, sweep, c);
}

#define AT(s, i, j, k) (s)[((i) * Y + (j)) * Z + (k)]

/* start: 0 = hot, 1 = cold. */
ORACLE_API void oracle3d_init(int8_t *s, int64_t X, int64_t Y, int64_t Z, uint64_t seed, int start)
{
#pragma omp parallel for schedule(static) if (X * Y * Z >= 32768)
    for (int64_t i = 0; i < X; ++i)
        for (int64_t j = 0; j < Y; ++j) {
            struct word_cache3 wc[2] = {{UINT64_MAX, {0}}, {UINT64_MAX, {0}}};
            for (int64_t k = 0; k < Z; ++k) {
                if (start == 1) {
                    AT(s, i, j, k) = 1;
                } else {
                    int c = (int)((i + j + k) & 1);
                    uint32_t x = cached_uniform3(&wc[c], plane_index3(Y, Z, i, j, k), seed, 0xFFFFFFFFu, c);
                    AT(s, i, j, k) = (x < 0x80000000u) ? 1 : -1;
                }
            }
        }
}

/* M = sum sigma, E = -sum over the 3N torus bonds. */
ORACLE_API void oracle3d_observe(const int8_t *s, int64_t X, int64_t Y, int64_t Z, int64_t *M, int64_t *E)
{
    int64_t m = 0, e = 0;
#pragma omp parallel for reduction(+ : m, e) schedule(static) if (X * Y * Z >= 32768)
    for (int64_t i = 0; i < X; ++i)
        for (int64_t j = 0; j < Y; ++j)
            for (int64_t k = 0; k < Z; ++k) {
                int64_t v = AT(s, i, j, k);
                m += v;
                e -= v * (AT(s, wrap3(i + 1, X), j, k) + AT(s, i, wrap3(j + 1, Y), k) + AT(s, i, j, wrap3(k + 1, Z)));
            }
    *M = m;
    *E = e;
}

/* One half-sweep of colour c.  words == NULL draws from Philox; otherwise
 * words[(i*Y + j)*Z + k] is the uniform word of site (i,j,k) (a test hook).
 * Returns the energy change, the sum of 2h over accepted flips. */
static int64_t half_sweep3d(int8_t *s, int64_t X, int64_t Y, int64_t Z, int c, const uint64_t T[3],
                            uint64_t seed, uint32_t sweep, const uint32_t *words)
{
    int64_t dE = 0;
#pragma omp parallel for reduction(+ : dE) schedule(static) if (X * Y * Z >= 32768)
    for (int64_t i = 0; i < X; ++i)
        for (int64_t j = 0; j < Y; ++j) {
            struct word_cache3 wc = {UINT64_MAX, {0}};
            for (int64_t k = 0; k < Z; ++k) {
                if (((i + j + k) & 1) != c) continue;
                int nn = AT(s, wrap3(i - 1, X), j, k) + AT(s, wrap3(i + 1, X), j, k)
                       + AT(s, i, wrap3(j - 1, Y), k) + AT(s, i, wrap3(j + 1, Y), k)
                       + AT(s, i, j, wrap3(k - 1, Z)) + AT(s, i, j, wrap3(k + 1, Z));
                int h = AT(s, i, j, k) * nn;
                uint32_t x = words ? words[(i * Y + j) * Z + k]
                                   : cached_uniform3(&wc, plane_index3(Y, Z, i, j, k), seed, sweep, c);
                if (oracle3d_accept(h, x, T)) {
                    AT(s, i, j, k) = (int8_t)(-AT(s, i, j, k));
                    dE += 2 * h;
                }
            }
        }
    return dE;
}

ORACLE_API int64_t oracle3d_half_sweep_words(int8_t *s, int64_t X, int64_t Y, int64_t Z, int c,
                                             const uint64_t T[3], const uint32_t *words)
{
    return half_sweep3d(s, X, Y, Z, c, T, 0, 0, words);
}

/* Exact h x w x d box (origin (i0, j0, k0), torus-wrapped) of the state after
 * sweeps sweep0 .. sweep0+nsweeps-1 from the start state, without the full lattice:
 * a site after one half-sweep depends only on itself and its six neighbours, so the
 * box grown by R = 2 nsweeps in every direction holds all that the box depends on.
 * Each half-sweep updates the sites of its colour whose neighbours are still exact
 * and shrinks the exact region by one; the uniforms are those of the sites' global
 * plane indices.  The grown box may exceed the torus: wrapped copies of a site then
 * evolve identically.  Returns -1 if the buffer cannot be had. */
ORACLE_API int oracle3d_window(int64_t X, int64_t Y, int64_t Z, double beta, uint64_t seed, int start,
                               int64_t sweep0, int64_t nsweeps, int64_t i0, int64_t j0, int64_t k0, int64_t h,
                               int64_t w, int64_t d, int8_t *out)
{
    uint64_t T[3];
    oracle3d_thresholds(beta, T);
    const int64_t R = 2 * nsweeps;
    const int64_t A = h + 2 * R, B = w + 2 * R, C = d + 2 * R;
    int8_t *buf = (int8_t *)malloc((size_t)(A * B * C));
    if (!buf) return -1;
#define BOX(a, b, c) buf[((a) * B + (b)) * C + (c)]
#pragma omp parallel for schedule(static) if (A * B * C >= 32768)
    for (int64_t a = 0; a < A; ++a)
        for (int64_t b = 0; b < B; ++b) {
            struct word_cache3 wc[2] = {{UINT64_MAX, {0}}, {UINT64_MAX, {0}}};
            for (int64_t c = 0; c < C; ++c) {
                int64_t gi = wrap3(i0 - R + a, X), gj = wrap3(j0 - R + b, Y), gk = wrap3(k0 - R + c, Z);
                if (start == 1) {
                    BOX(a, b, c) = 1;
                } else {
                    int col = (int)((gi + gj + gk) & 1);
                    uint32_t x = cached_uniform3(&wc[col], plane_index3(Y, Z, gi, gj, gk), seed, 0xFFFFFFFFu, col);
                    BOX(a, b, c) = (x < 0x80000000u) ? 1 : -1;
                }
            }
        }
    for (int64_t t = 0; t < 2 * nsweeps; ++t) {
        uint32_t sweep = (uint32_t)(sweep0 + t / 2);
        int col = (int)(t & 1);
        int64_t lo = t + 1;
#pragma omp parallel for schedule(static) if (A * B * C >= 32768)
        for (int64_t a = lo; a < A - lo; ++a)
            for (int64_t b = lo; b < B - lo; ++b) {
                struct word_cache3 wc = {UINT64_MAX, {0}};
                for (int64_t c = lo; c < C - lo; ++c) {
                    int64_t gi = wrap3(i0 - R + a, X), gj = wrap3(j0 - R + b, Y), gk = wrap3(k0 - R + c, Z);
                    if (((gi + gj + gk) & 1) != col) continue;
                    int nn = BOX(a - 1, b, c) + BOX(a + 1, b, c) + BOX(a, b - 1, c) + BOX(a, b + 1, c) +
                             BOX(a, b, c - 1) + BOX(a, b, c + 1);
                    int hh = BOX(a, b, c) * nn;
                    uint32_t x = cached_uniform3(&wc, plane_index3(Y, Z, gi, gj, gk), seed, sweep, col);
                    if (oracle3d_accept(hh, x, T)) BOX(a, b, c) = (int8_t)(-BOX(a, b, c));
                }
            }
    }
    for (int64_t a = 0; a < h; ++a)
        for (int64_t b = 0; b < w; ++b)
            for (int64_t c = 0; c < d; ++c) out[(a * w + b) * d + c] = BOX(a + R, b + R, c + R);
#undef BOX
    free(buf);
    return 0;
}

/* Sweeps sweep0 .. sweep0+nsweeps-1 (black then white) on s; M[k], E[k] after
 * each sweep when non-NULL.  check != 0 also carries E incrementally and compares
 * it with the recomputed value after every half-sweep; returns the mismatches. */
ORACLE_API int64_t oracle3d_run(int8_t *s, int64_t X, int64_t Y, int64_t Z, double beta, uint64_t seed,
                                int64_t sweep0, int64_t nsweeps, int64_t *M, int64_t *E, int check)
{
    uint64_t T[3];
    oracle3d_thresholds(beta, T);
    int64_t mism = 0, m0 = 0, e_inc = 0;
    if (check) oracle3d_observe(s, X, Y, Z, &m0, &e_inc);
    for (int64_t n = 0; n < nsweeps; ++n) {
        uint32_t sweep = (uint32_t)(sweep0 + n);
        for (int c = 0; c < 2; ++c) {
            int64_t dE = half_sweep3d(s, X, Y, Z, c, T, seed, sweep, NULL);
            if (check) {
                int64_t m, e;
                e_inc += dE;
                oracle3d_observe(s, X, Y, Z, &m, &e);
                if (e != e_inc) ++mism;
            }
        }
        if (M || E) {
            int64_t m, e;
            oracle3d_observe(s, X, Y, Z, &m, &e);
            if (M) M[n] = m;
            if (E) E[n] = e;
        }
    }
    return mism;
}

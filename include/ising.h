/*
 * ising.h -- C ABI of the GB300 checkerboard Metropolis library (libising_gb300.so).
 *
 * The library simulates the 2D nearest-neighbour Ising model
 *     H(sigma) = -J sum_<ij> sigma_i sigma_j - mu sum_i sigma_i,  mu = 0, J = 1,
 * on an L x L torus (paper Sec. 3) with the checkerboard Metropolis-within-Gibbs
 * sweep of Sec. 3.1: every black site (i+j even) is updated with the white sites
 * fixed, then every white site with the black sites fixed; a site with
 * h = sigma_i * nn(i) flips with probability min{1, exp(-2 beta h)}.
 * One "sweep" is one black plus one white half-sweep (the unit of the paper's
 * flips/ns, Sec. 4.2).
 *
 * Determinism.  The chain is a pure function of (L, beta, seed, start state,
 * sweep count):
 *   - uniform of site (i,j) of colour c in sweep s: with plane index
 *     p = i*(L/2) + (j>>1), plane word g = p >> 5 and bit b = p & 31,
 *     U = sum_k bit_b(R_k) 2^(31-k), where R_k (k = 0..31) is output word (k & 3)
 *     of Philox4x32-10 (Salmon et al., SC'11) with key (seed lo32, seed hi32) and
 *     counter (s, q lo32, c, q hi32), q = 8g + (k >> 2): the 32 random words of a
 *     plane word are the bit planes of its 32 uniforms, R_0 the top one;
 *   - flip iff h <= 0, or U < T_h with T_h = min(2^32, ceil(exp(-2 beta h) 2^32))
 *     computed on the host in FP64 (see ising_thresholds);
 *   - hot start: sigma = +1 iff the uniform drawn with s = 0xFFFFFFFF is < 2^31;
 *     cold start: all +1.
 *   Both kernels (bit-packed and int8) produce the same lattice bit for bit.
 *
 * Observables after each sweep: M = sum_i sigma_i and E = H(sigma) as exact
 * 64-bit integers (Sec. 4.1 magnetisation; E from the Sec. 3 Hamiltonian).
 *
 * Conventions for every function:
 *   - returns ISING_OK (0) or a negative ISING_E* code; outputs are written only
 *     on ISING_OK; ising_last_error() returns a thread-local message for the
 *     last failure on the calling thread;
 *   - host pointers are caller-owned and only read/written during the call;
 *   - handles own all device memory they allocate (cudaMalloc) and release it in
 *     the matching *_free; a handle must not be used from two threads at once,
 *     distinct handles may;
 *   - work is enqueued on the handle's CUDA stream; functions that return data
 *     to the host synchronise that stream.
 */
#ifndef ISING_GB300_H
#define ISING_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISING_OK 0
#define ISING_EINVAL (-1)   /* bad argument (size, beta, index, null pointer) */
#define ISING_ENOMEM (-2)   /* device allocation or HBM budget exhausted */
#define ISING_ECUDA (-3)    /* CUDA runtime error (message in ising_last_error) */
#define ISING_ETIMEOUT (-4) /* a kernel's bounded wait expired; results invalid */
#define ISING_EBUSY (-5)    /* slot table full */

#define ISING_HOT 0
#define ISING_COLD 1

#define ISING_PACKED 0 /* multi-spin-coded black/white bit planes; L % 64 == 0 */
#define ISING_INT8 1   /* row-major int8 +1/-1 lattice; L % 8 == 0 */

typedef struct ising_s *ising_t;
typedef struct ising_batch_s *ising_batch_t;

/* Thread-local description of the last error on this thread ("" if none). */
const char *ising_last_error(void);

/* Library version string. */
const char *ising_version(void);

/*
 * Acceptance thresholds (Sec. 3.1 acceptance rule, Algorithm 1-2's
 * exp(-2 nn sigma) with beta restored): T[0] for h = 2, T[1] for h = 4,
 * T_h = min(2^32, ceil(exp(-2 beta h) * 2^32)) in FP64 with the host libm exp.
 * A site's 32-bit uniform U accepts iff U < T_h.  beta must be finite and >= 0.
 * Host-only; needs no GPU.  Errors: EINVAL.
 */
int ising_thresholds(double beta, uint64_t T[2]);

/* ------------------------------------------------------------------------
 * Single lattice
 * ---------------------------------------------------------------------- */

/*
 * Creates a lattice of side L at inverse temperature beta with Philox seed
 * `seed`: hot start, bit-packed kernel, default stream.  Equivalent to
 * ising_init_ex(out, L, beta, seed, ISING_HOT, ISING_PACKED, NULL).
 * Paper: Sec. 3 (the L x L torus, H with mu = 0, J = 1, inverse temperature beta).
 */
int ising_init(ising_t *out, int64_t L, double beta, uint64_t seed);

/*
 * Paper: Sec. 3 (the torus and H), Sec. 3.2 (the lattice held as compact colour
 * sub-lattices, here bit planes).
 * start: ISING_HOT or ISING_COLD.  kernel: ISING_PACKED (L % 64 == 0, 64 <= L <=
 * 1048576 when L % 256 == 0 -- rows longer than 4,264 words are swept in 2-row
 * column blocks -- else L <= 102336, so that a double-buffered tile of whole rows
 * fits one 100 KB shared-memory stage) or ISING_INT8 (L % 8 == 0, 8 <= L <= 131072).  stream: a cudaStream_t
 * on which all of this handle's work is enqueued (the caller keeps it alive
 * until ising_free); NULL makes the handle create and own a non-blocking stream.  Device memory: packed L*L/8
 * bytes, int8 L*L bytes, plus 16 bytes of history per sweep (grown on demand).
 * Errors: EINVAL (L, beta, start, kernel), ENOMEM, ECUDA.
 */
int ising_init_ex(ising_t *out, int64_t L, double beta, uint64_t seed, int start, int kernel, void *stream);

/*
 * Paper: Sec. 3.1 (one sweep = the black then the white half of the checkerboard
 * kernel, each site flipped with probability min{1, exp(-2 beta h)}).
 * Enqueues n sweeps (n >= 0) on the handle's stream; returns without waiting.
 * The sweep counter advances by n (total must stay below 2^32 - 1) and the
 * per-sweep (M, E) history grows by n entries.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int ising_sweep(ising_t h, int64_t n);

/*
 * Paper: Sec. 4.1 (magnetisation) and Sec. 3 (E = H(sigma)).
 * Current M and E (after the last sweep; the start state if none) and the
 * number of sweeps done.  Synchronises.  Any output pointer may be NULL.
 * Errors: EINVAL, ECUDA, ETIMEOUT.
 */
int ising_observables(ising_t h, int64_t *M, int64_t *E, int64_t *sweeps_done);

/*
 * Paper: Sec. 4.1 (one (M, E) sample per sweep, the series its moments average).
 * Copies history entries first .. first+count-1 (sweep indices, 0-based) into
 * the caller's arrays M[count] and E[count] (either may be NULL).  Synchronises.
 * Errors: EINVAL (range beyond sweeps done), ECUDA, ETIMEOUT.
 */
int ising_history(ising_t h, int64_t first, int64_t count, int64_t *M, int64_t *E);

/*
 * Sec. 4.1 observables over samples s = burn_in .. sweeps_done-1 (the paper drops
 * the first 10 % as burn-in), from exact integer sums on the device, evaluated in
 * FP64 once: *abs_m = <|m|>, *m2 = <m^2>, *m4 = <m^4>, *e = <e> (E/N) and
 * *binder = U4 = 1 - <m^4>/(3 <m^2>^2), m = M/N.  Any output may be NULL.
 * Synchronises.  Errors: EINVAL (null handle, no samples after burn_in), ECUDA.
 */
int ising_moments(ising_t h, int64_t burn_in, double *abs_m, double *m2, double *m4, double *e, double *binder);

/*
 * As ising_moments, with <e^2> and the exact sums as well: out[0] = <|m|>,
 * out[1] = <m^2>, out[2] = <m^4>, out[3] = <e>, out[4] = <e^2>, out[5] = U4.
 * sums (may be NULL) receives the 11 exact 64-bit limbs: sum|M|, sum M^2 (2
 * limbs, little-endian), sum M^4 (4), sum E (2, two's complement), sum E^2 (2).
 * Synchronises.  Errors: EINVAL (no samples), ECUDA.
 */
int ising_moments_ex(ising_t h, int64_t burn_in, double out[6], uint64_t sums[11]);

/* Copies the lattice into out[L*L] (row-major, +1 / -1).  Synchronises.
 * Paper: Sec. 3 (the spin configuration sigma). */
int ising_get_lattice(ising_t h, int8_t *out);

/*
 * Copies rows row0 .. row0+nrows-1 of the lattice into out[nrows*L] (row-major,
 * +1 / -1; for a cube the rows are r = i*L + j, L sites each), so that a window of a
 * lattice too large for host memory can be read.  Caller-owned out.  Synchronises.
 * Errors: EINVAL (rows outside the lattice, null out), ECUDA, ETIMEOUT.
 */
int ising_get_rows(ising_t h, int64_t row0, int64_t nrows, int8_t *out);

/*
 * Replaces the lattice by in[L*L] (row-major, each entry +1 or -1; other values
 * are EINVAL).  Does not change the sweep counter.  Synchronises.
 * Paper: Sec. 3 (the spin configuration sigma).
 */
int ising_set_lattice(ising_t h, const int8_t *in);

/*
 * Packed handles only: copy the bit planes to / from host arrays of L*L/64
 * uint32 words each (row i, word w at index i*(L/64) + w; bit b is site
 * (i, 2(32w+b) + ((i+c)&1)) of colour c; 1 = +1).  Synchronises.
 */
int ising_get_planes(ising_t h, uint32_t *black, uint32_t *white);
int ising_set_planes(ising_t h, const uint32_t *black, const uint32_t *white);

/*
 * Checkpoint: ising_state_bytes gives the size of the blob; ising_save writes
 * (L, beta, seed, kernel, sweeps done, lattice, history) into buf; ising_load
 * creates a new handle that continues the same chain bit for bit.  ising_load
 * returns ISING_EINVAL, before creating any handle or device memory, for a
 * buffer that is not a checkpoint, is shorter than its header says, or whose
 * kernel, start or sweep count is out of range; *out is then left unchanged.
 */
int ising_state_bytes(ising_t h, int64_t *bytes);
int ising_save(ising_t h, void *buf, int64_t bytes);
int ising_load(ising_t *out, const void *buf, int64_t bytes, void *stream);

/* Waits for the handle's work; reports ETIMEOUT if a kernel gave up. */
int ising_synchronize(ising_t h);

/*
 * Kernels compiled for a lattice's thresholds.  The acceptance test compares each
 * site's uniform with T_h bit plane by bit plane (Sec. 3.1's acceptance rule as an
 * integer comparison); compiled with T_2 and T_4 as constants, each plane needs one
 * to three logic operations instead of four, and the whole sweep about a fifth less
 * time at the critical point.  A packed single handle of L > 256 can have its sweep
 * kernel compiled that way (NVRTC, a few seconds, once per threshold pair and
 * process) when it is created; the chain is the same bit for bit.
 *
 * ising_set_specialize sets the process-wide mode for handles created afterwards:
 * ISING_SPECIALIZE_OFF (never), ISING_SPECIALIZE_AUTO (default: sides L >= 16384,
 * where the compile is repaid within some thousands of sweeps) or
 * ISING_SPECIALIZE_ALWAYS.  Where NVRTC or the compile is unavailable the handle
 * uses the built-in kernel.  Errors: EINVAL (mode).
 *
 * ising_specialized: *specialized = 1 when the handle sweeps with a specialised
 * kernel, else 0; note (may be NULL) receives a NUL-terminated reason of at most
 * len bytes.  Host-only, does not synchronise.  Errors: EINVAL (null handle).
 */
#define ISING_SPECIALIZE_OFF 0
#define ISING_SPECIALIZE_AUTO 1
#define ISING_SPECIALIZE_ALWAYS 2
int ising_set_specialize(int32_t mode);
int ising_specialized(ising_t h, int32_t *specialized, char *note, int64_t len);

/*
 * Batches: while every lattice of a batch has the same thresholds, the batch sweeps
 * with the multi-lattice kernel compiled for them (mode ALWAYS, or AUTO once the
 * batch holds at least 16384^2 sites); a lattice of another temperature brings back
 * the built-in kernel (captured graphs are re-captured).  *specialized = 1 while the
 * compiled kernel is in use.  Host-only.  Errors: EINVAL (null argument).
 */
int ising_batch_specialized(ising_batch_t b, int32_t *specialized);

/*
 * Cluster-resident batches.  While every lattice of a batch has the same side
 * L <= 4096 (whole-row tiles), the batch can keep each lattice in the shared
 * memory of one thread-block cluster for a whole run (CTA r of a cluster of C
 * holds rows [r L/C, (r+1) L/C), reading its halo rows from the neighbouring CTAs'
 * shared memory after every half-sweep) and run up to 4,096 sweeps per launch; C
 * is the largest power of two (at most 16, at least 16 rows per CTA) for which
 * every lattice's cluster can be resident at once (else 1, the lattices then
 * running in waves).  The chain is the tiled kernel's, bit for bit.
 * mode ISING_CLUSTER_OFF keeps the batch on the tiled kernel; ISING_CLUSTER_AUTO
 * (the default) takes the cluster form when its estimated rate (about 22 sites/ns
 * per SM its CTAs occupy) beats the tiled kernel's (about 25.7 sites/ns per SM,
 * halved at 5e7 sites per sweep): many small lattices, or a few of L <= 2048;
 * ISING_CLUSTER_ALWAYS whenever the lattices fit.
 * ising_batch_cluster_size gives the C in use (0: the tiled kernel).  Host-only;
 * the mode is re-applied whenever lattices are added or removed.
 * Paper: Sec. 3.1 (the schedule), Sec. 4.1 (scans of small lattices).
 * Errors: EINVAL (null argument, mode not 0-2).
 */
#define ISING_CLUSTER_OFF 0
#define ISING_CLUSTER_AUTO 1
#define ISING_CLUSTER_ALWAYS 2
int ising_batch_set_cluster(ising_batch_t b, int32_t mode);
int ising_batch_cluster_size(ising_batch_t b, int32_t *cluster_size);

/* Releases the handle and its device memory (NULL is a no-op).  Paper: none (resource
 * management of the Sec. 3 lattice). */
int ising_free(ising_t h);

/* ------------------------------------------------------------------------
 * Three-dimensional lattice.  Sec. 3 writes the Hamiltonian for a
 * d-dimensional hypercubic lattice and the Conclusion states that the
 * checkerboard algorithm carries over to three dimensions; these handles run
 * that generalisation on the cubic L x L x L torus: colour c = (i+j+k) & 1
 * (black first), nn = sum of the six neighbours, h = sigma * nn, flip iff
 * h <= 0 or the site's uniform is below T_h, h = 2, 4, 6.  E = H(sigma)
 * over the 3N bonds.  Uniform of site (i,j,k): as in 2D from plane index
 * p = (i*L + j)*(L/2) + (k>>1) -- the 2D keying with row index i*L + j.  Hot
 * start as in 2D.
 * ---------------------------------------------------------------------- */

/*
 * T[0], T[1], T[2] for h = 2, 4, 6: T_h = min(2^32, ceil(exp(-2 beta h) 2^32))
 * in host FP64 (T[0], T[1] equal ising_thresholds).  Host-only.  Errors: EINVAL.
 */
int ising_thresholds3d(double beta, uint64_t T[3]);

/*
 * Creates a bit-packed cubic lattice of side L (L % 64 == 0, 64 <= L <= 8192):
 * device memory L^3/8 bytes of planes plus 16 bytes of history per sweep.
 * start and stream as in ising_init_ex.  The handle works with ising_sweep,
 * ising_observables, ising_history, ising_moments[_ex] (N = L^3), ising_get_lattice
 * (out[L^3], index (i*L + j)*L + k), ising_get_planes / ising_set_planes (L*L
 * rows of L/64 words each per colour, row i*L + j; bit b of word w is the site
 * (i, j, 2(32w+b) + ((i+j+c)&1))), the checkpoint calls, ising_synchronize and
 * ising_free; ising_set_lattice returns EINVAL.
 * Errors: EINVAL (L, beta, start), ENOMEM, ECUDA.
 */
int ising_init3d(ising_t *out, int64_t L, double beta, uint64_t seed, int start, void *stream);

/* ------------------------------------------------------------------------
 * Batch: many packed lattices of uneven L and beta swept by one persistent
 * launch per half-sweep (the single-device analogue of the paper's replicated
 * program, Sec. 5.1), optionally replayed from a captured CUDA graph.
 * ---------------------------------------------------------------------- */

/*
 * Creates a batch of `count` packed lattices from caller-owned host arrays of
 * length count (read during the call only): lattice k has side L[k] (the sizes
 * ising_init_ex accepts for ISING_PACKED), inverse temperature beta[k] (finite,
 * >= 0), Philox seed seed[k] and start[k] (ISING_HOT or ISING_COLD); it is slot k
 * of the batch.  Paper: Sec. 3 (each lattice), Sec. 5.1 (many independent
 * simulations run as one replicated program, here one launch).
 * The lattices have no sweep limit: every ising_batch_run sweeps all of them, and
 * their (M, E) histories live outside the planes' arena and grow (doubling) when a
 * run needs room.  Tiles: the tallest whole-row tile of at most 8,192 words for each
 * lattice when the batch then holds at least two tiles per CTA of its persistent grid,
 * else the built-in shapes; 256-thread CTAs (512 when a side is at least 16,384), a
 * stream the batch owns.
 * EINVAL, before any device work, for a null array, count outside 1 .. 2^20, or
 * any bad L, beta or start (the message names the lattice).  ENOMEM, ECUDA.
 */
int ising_batch_create(ising_batch_t *out, int32_t count, const int64_t *L, const double *beta,
                       const uint64_t *seed, const int32_t *start);

/*
 * Creates an empty batch that can hold up to `capacity` lattices of side <=
 * max_L with `arena_bytes` of device memory for planes and histories (the HBM
 * budget; allocation beyond it is ENOMEM); lattices join with ising_batch_add and
 * run at most the sweeps they were admitted for.  threads: CTA size of the sweep
 * kernel (128, 256 or 512; 0 = 256).  stream as in ising_init_ex.
 * EINVAL, before any device work, unless 1 <= capacity <= 2^20, max_L is a
 * multiple of 64 in 64 .. 2^20 and arena_bytes >= 256.
 */
int ising_batch_create_ex(ising_batch_t *out, int32_t capacity, int64_t max_L, int64_t arena_bytes, int32_t threads,
                          void *stream);

/*
 * Adds a packed lattice (L % 64 == 0, L <= max_L, and within the sizes
 * ising_init_ex accepts for ISING_PACKED) that will run `sweeps`
 * sweeps at most (its history capacity).  tile_rows: rows per tile (a power of
 * two from 4 to 256 dividing L, or 2 when L % 256 == 0, whose shared-memory stage
 * fits in 100 KB; 0 = built-in choice).
 * Writes the slot index to *idx.
 * Enqueues the start state.  Errors: EINVAL, ENOMEM (arena), EBUSY (slots).
 */
int ising_batch_add(ising_batch_t b, int64_t L, double beta, uint64_t seed, int32_t start, int64_t sweeps,
                    int32_t tile_rows, int32_t *idx);

/*
 * As ising_batch_add with the tile's width as well: tile_words = L/64 (whole rows),
 * 0 (built-in: whole rows when they fit a stage, else column blocks), or a column
 * block of tile_words words of each of tile_rows rows (tile_words a multiple of 4
 * dividing L/64, below it; L % 256 == 0; tile_rows a power of two from 2 to 256
 * dividing L, 0 = 2), each source row staged with 4 halo words on either side.  The
 * chain does not depend on the tile shape.  Errors as ising_batch_add, and EINVAL
 * for a block that is not of that form or whose stage exceeds the batch's (the
 * largest built-in stage of its sides).
 */
int ising_batch_add_tiled(ising_batch_t b, int64_t L, double beta, uint64_t seed, int32_t start, int64_t sweeps,
                          int32_t tile_rows, int32_t tile_words, int32_t *idx);

/* Frees a slot and its arena memory (after the stream's pending work). */
int ising_batch_remove(ising_batch_t b, int32_t idx);

/*
 * Enqueues `sweeps` sweeps of every lattice in the batch; a lattice admitted with
 * ising_batch_add stops at its own sweep limit.  graph_sweeps (the use_graph
 * switch) > 0: capture graph_sweeps sweeps into a CUDA graph once per distinct
 * graph_sweeps (a few are kept) and replay it sweeps / graph_sweeps times (sweeps
 * must be a multiple, else EINVAL); 0: plain launches.  Admitting, removing and
 * running lattices enqueue work without waiting for the stream's earlier sweeps
 * (batches of more than 7,679 lattices wait when the tile table changes).
 * Paper: Sec. 3.1 (the sweep), Sec. 5.1.
 */
int ising_batch_run(ising_batch_t b, int64_t sweeps, int32_t graph_sweeps);

/* Per-lattice sweeps done (synchronises). */
int ising_batch_sweeps_done(ising_batch_t b, int32_t idx, int64_t *sweeps_done);

/*
 * Sweeps done of slots 0 .. n-1 in one device-to-host copy (-1 for a free
 * slot); n <= capacity.  Synchronises.
 */
int ising_batch_progress(ising_batch_t b, int64_t *sweeps_done, int32_t n);

/*
 * Without waiting: enqueues on the batch's stream a kernel that writes, for slot
 * idx[k] (k < n), its sweeps done, M and E after its last sweep (0, 0 before any)
 * to out[3k], out[3k+1], out[3k+2], as they stand once the work enqueued before it
 * has run.  out: device-accessible memory of 3n int64 (device memory, or page-locked
 * host memory the caller polls after recording an event on the stream); idx is read
 * during the call only.  A slot may be removed right after the call (its memory is
 * reused only by later work of the stream).  For a serving loop that keeps sweeps in
 * flight while it collects results.  Errors: EINVAL (n, a free or bad slot), ECUDA.
 */
int ising_batch_gather(ising_batch_t b, int32_t n, const int32_t *idx, int64_t *out);

/*
 * Slot idx: current M and E (the start state before any sweep; Sec. 4.1, Sec. 3);
 * the _ex form also gives the sweeps done.  History entries first .. first+count-1;
 * Sec. 4.1 moments over samples burn_in .. sweeps_done-1 (as ising_moments_ex); the
 * lattice as L*L int8 +1/-1.  All synchronise.
 */
int ising_batch_observables(ising_batch_t b, int32_t idx, int64_t *M, int64_t *E);
int ising_batch_observables_ex(ising_batch_t b, int32_t idx, int64_t *M, int64_t *E, int64_t *sweeps_done);
int ising_batch_history(ising_batch_t b, int32_t idx, int64_t first, int64_t count, int64_t *M, int64_t *E);
int ising_batch_moments(ising_batch_t b, int32_t idx, int64_t burn_in, double out[6], uint64_t sums[11]);
int ising_batch_get_lattice(ising_batch_t b, int32_t idx, int8_t *out);

/* Arena bytes in use and slots in use. */
int ising_batch_usage(ising_batch_t b, int64_t *arena_used, int32_t *slots_used);

/* Waits for the batch's work; ETIMEOUT if a kernel gave up. */
int ising_batch_synchronize(ising_batch_t b);

int ising_batch_free(ising_batch_t b);

/*
 * Times sweeps of packed lattices of side L for each candidate (tile_rows a
 * power of two from 2 to 256 accepted by ising_batch_add; threads 256 or 512),
 * using enough copies of the lattice (up to 2^26 sites or 64) to give every SM
 * work, each candidate timed twice over about 2^32 site updates (16 to 256 sweeps),
 * and returns the fastest in *tile_rows, *threads and its time per sweep of one
 * lattice in *ms.  Whole-row tiles only: EINVAL for L whose rows need column blocks
 * (L > 272896).  Uses its own scratch batch.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int ising_autotune(int64_t L, int32_t *tile_rows, int32_t *threads, double *ms);

/* ------------------------------------------------------------------------
 * Device-side building blocks on caller-owned device memory (for tests and
 * for callers that manage memory themselves).  All pointers are device
 * pointers; work is enqueued on `stream` and not waited for.
 * ---------------------------------------------------------------------- */

/*
 * Philox4x32-10 of counters (ctr0 + k as a 64-bit value in words 0-1, ctr[2],
 * ctr[3]) for k = 0 .. nblocks-1 under key `key`; out[4*nblocks] (device).
 */
int ising_dev_philox(uint64_t key, const uint32_t ctr[4], int64_t nblocks, uint32_t *out, void *stream);

/*
 * Packed sweeps of caller-owned lattices with no device allocation.  The paper
 * has no counterpart; this serves callers that cannot call cudaMalloc -- code
 * running while a CUDA graph is being captured, plugins confined to another
 * runtime's memory pool, loops whose memory must be fixed after start-up.
 *
 * count lattices (1 <= count <= 64; more is ISING_EINVAL).  For lattice k:
 * black[k], white[k] are device pointers to its two bit planes in the layout of
 * ising_get_planes (L[k]*L[k]/64 uint32 words each, updated in place); L[k] %
 * 64 == 0, 64 <= L[k], L[k] <= 163840 when L[k] % 256 == 0 and L[k] <= 102336
 * otherwise (4-row tiles must fit a 100 KB stage); beta[k] finite and >= 0; seed[k] its Philox key;
 * me[k] a device array of 2*nsweeps int64 that receives (M, E) after each of the
 * sweeps first_sweep .. first_sweep+nsweeps-1 (M at [2s], E at [2s+1], s counted
 * from first_sweep).  me[k] need not be cleared: each sweep overwrites its pair
 * (the black half-sweep stores the pair's starting value, the white half-sweep adds
 * the counts), whatever the array held before.  The host arrays black, white, L,
 * beta, seed, me are read during the call only.  The chain is the one ising_sweep
 * produces: calling with first_sweep = n continues n sweeps done earlier, bit for
 * bit.  The sweep numbers (and so the random numbers) of a call are fixed by its
 * first_sweep: work enqueued by one call always repeats sweeps first_sweep ..
 * first_sweep+nsweeps-1, and a chain goes on only through a call with the next
 * first_sweep.
 *
 * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream).
 * wait != 0: the call synchronises the stream and returns ISING_ETIMEOUT if a
 * bounded wait in the sweep kernel expired (ISING_ECUDA for any other status the
 * kernel reports); a stream that is being captured cannot be synchronised, so
 * wait != 0 on one is ISING_EINVAL before any work.  wait == 0: it returns at once.
 *
 * Scratch (64 descriptors, tile table, count and status word: 5,392 bytes) is a file-scope
 * __device__ array that every GPU loading this library holds until exit; no
 * call allocates or frees device memory.  The first call on a device looks up
 * that array's address (cudaGetSymbolAddress) and sets the kernel's
 * shared-memory limit: make it before any stream capture.  All calls share the
 * scratch, which keeps the last call's contents (each call rewrites it and
 * clears the status word first), so calls whose work overlaps on the GPU race.
 * Errors: EINVAL, ECUDA, ETIMEOUT (message in ising_last_error).
 */
int ising_sweep_packed_noalloc(int32_t count, uint32_t *const *black, uint32_t *const *white, const int64_t *L,
                               const double *beta, const uint64_t *seed, int64_t first_sweep, int64_t nsweeps,
                               int64_t *const *me, void *stream, int32_t wait);

/*
 * Failure-detection self-test of the sweep kernel's bounded waits.  Launches one
 * half-sweep of a 256 x 256 lattice whose tile barriers expect 16 bytes that are
 * never sent, with each wait bounded by wait_cycles SM clocks (>= 1000), then
 * writes the status the host read back to *observed (ISING_ETIMEOUT when the
 * kernel gave up as designed) and runs one normal sweep to show the context is
 * still usable.  Returns ISING_OK when that sweep succeeded.  No fault, trap or
 * unbounded wait is involved.  Not part of the paper: a test hook.
 */
int ising_selftest_timeout(int64_t wait_cycles, int *observed);

/*
 * Integer-pipe throughput of this GPU, the denominator of the sweep's ALU
 * roofline: out[0] = 32x32->64 multiplies (both halves used, as in a Philox
 * round) per SM per clock; out[1] = ALU ops (3-input XOR, funnel shift) per SM
 * per clock.  Runs two short compute-only kernels and synchronises the device.
 * Not part of the paper: measurement support.  Errors: ENOMEM, ECUDA.
 */
int ising_probe_int_rates(double out[2]);

#ifdef __cplusplus
}
#endif

#endif /* ISING_GB300_H */

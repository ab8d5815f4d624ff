/*
 * ising.h -- C ABI of the GB300 multi-spin Ising Metropolis library.
 *
 * The library simulates the 2D square Ising model of Hassani & Rafibakhsh,
 * "Parallelization and implementation of multi-spin Monte Carlo simulation of
 * 2D square Ising model using MPI and C++" (arXiv:1811.04384):
 *   Eq. 1      H = -J sum_<mn> s_m s_n, nearest neighbours, periodic
 *              boundaries, J = 1, K = 1, no field;
 *   Sec. 2     Metropolis: a flip with dE <= 0 is accepted, otherwise with
 *              probability exp(-dE/KT);
 *   Sec. 3     multi-spin coding: 3-bit fields (000 = down, 001 = up), 21
 *              spins per 64-bit word, bit 63 always zero;
 *   Eq. 3,     the neighbour count of every field from XORs of whole words,
 *   Table 1    and dE = 8 - 4a for a anti-aligned neighbours;
 *   Sec. 5.3   the energy as the sum over right and down bonds;
 *   Eq. 2      averages of the per-sweep energies.
 *
 * Conventions that the paper leaves open and this library fixes:
 *   - a lattice is L x L, L even, 4 <= L <= 32768; site (i, j), row i,
 *     column j, colour c = (i + j) & 1;
 *   - sweep t (t = 1, 2, ...) updates colour 0, then colour 1;
 *   - the draw of site (i, j) at sweep t is output word (i & 3) of
 *     Philox4x32-10 (Salmon et al., SC'11) with key (lo32(seed), hi32(seed))
 *     and counter (i >> 2, j >> 1, lo32(t), hi32(t) << 1 | c);
 *   - a site with a >= 2 anti-aligned neighbours always flips; a site with
 *     a in {0, 1} flips iff draw < thr[a], thr[a] = floor(2^32 exp(-(8 - 4a)
 *     beta)) computed in IEEE double on the host;
 *   - a hot start sets s = +1 iff the site's draw at t = 0 is below 2^31;
 *   - E = -sum s_ij (s_i+1,j + s_i,j+1) and M = sum s_ij, both exact int64.
 *
 * Return values: ISING_OK (0) on success, a negative ISING_E* code otherwise;
 * ising_strerror() names it.  No function aborts the process.
 *
 * Memory and threads: every pointer argument named host_* or documented as a
 * host array is caller-owned host memory; the library owns all device memory
 * it allocates.  A handle is not thread-safe: one thread at a time.  All work
 * is ordered on the handle's CUDA stream (the legacy default stream unless
 * ising_set_stream() chose another); functions that return values to the host
 * synchronise that stream.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ISING_OK = 0,
    ISING_EINVAL = -1,    /* bad argument: odd or out-of-range L, beta < 0 or NaN,
                             NULL pointer, buffer too small, bad count */
    ISING_ENOMEM = -2,    /* device or host allocation failed */
    ISING_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    ISING_ETIMEOUT = -4,  /* a bounded wait gave up: ising_server_wait, or a wait between
                             clusters of a cluster-path launch (each gives up after 1 s) */
    ISING_EBUSY = -5,     /* no free slot / budget (server admission) */
    ISING_ENOTFOUND = -6, /* unknown request id */
    ISING_EINTERNAL = -7  /* a host exception inside the server's worker thread
                             (an allocation failure, or ising_server_inject_fault) */
};

typedef struct ising_lattice ising_lattice;   /* opaque, library-owned */

/* Text for an ISING_* code (static storage; never NULL). */
const char *ising_strerror(int code);

/* The last CUDA failure seen by this thread ("call: message"), or "". */
const char *ising_last_cuda_error(void);

/* Device bytes one lattice of side L occupies inside the library: two colour
 * arrays of L rows x pitch 64-bit words (pitch = words per colour-row rounded
 * up to even) plus the energy/magnetisation count slots.  0 if L is invalid. */
size_t ising_bytes_required(int32_t L);

/* Create a lattice of side L with Philox seed `seed`: all spins +1, t = 0,
 * beta = 0.  Allocates its device memory with cudaMalloc on the current
 * device.  *out receives the handle.  Errors: EINVAL (L odd, < 4, > 32768,
 * out NULL), ENOMEM, ECUDA. */
int ising_create(int32_t L, uint64_t seed, ising_lattice **out);

/* As ising_create, but the lattice lives in caller-owned device memory
 * dev_buf of `bytes` bytes (>= ising_bytes_required(L), 256-byte aligned),
 * which must stay valid until ising_destroy; `stream` (a cudaStream_t, may be
 * NULL) becomes the handle's stream.  Errors: EINVAL (also for a small or
 * misaligned buffer), ECUDA. */
int ising_create_on(int32_t L, uint64_t seed, void *dev_buf, size_t bytes,
                    void *stream, ising_lattice **out);

/* The paper's own word layout (Sec. 3, Fig. 1-2) as an alternative:
 * ISING_LAYOUT_COLUMN_INTERLEAVED stores the lattice as N x L words,
 * N = L / 21, word S(I, J) holding s(I + kN, J) in field k, with the
 * one-field rotation of the neighbour word across the top and bottom word
 * rows, and updates it with the arithmetic form of Eq. 3.  Needs L % 84 == 0
 * (the paper's L = 21N with N divisible by 4, e.g. 1008 and 2016).  The
 * chain, E and M are identical to the default row-packed layout
 * (ISING_LAYOUT_ROW_PACKED), which works for any even L.  Calls that expose
 * the row-packed words (ising_get_words, ising_set_words, ising_layout,
 * ising_device_words, ising_set_tiling, the on-chip path) return EINVAL on
 * an interleaved lattice. */
#define ISING_LAYOUT_ROW_PACKED 0
#define ISING_LAYOUT_COLUMN_INTERLEAVED 1
int ising_create_layout(int32_t L, uint64_t seed, int32_t layout, ising_lattice **out);

/* Release the handle and every device buffer the library allocated for it
 * (not a caller-owned dev_buf).  NULL is accepted. */
int ising_destroy(ising_lattice *h);

/* Hot start (Sec. 5.1: every spin up or down at random): s(i,j) = +1 iff the
 * site's Philox draw at t = 0 is below 2^31.  Resets t to 0.  Asynchronous on
 * the stream.  Errors: EINVAL (NULL), ECUDA. */
int ising_init_hot(ising_lattice *h);

/* Cold start: every spin = `spin` (+1 or -1, else EINVAL).  Resets t to 0.
 * Asynchronous on the stream.  Errors: EINVAL, ECUDA. */
int ising_init_cold(ising_lattice *h, int8_t spin);

/* Set the inverse temperature (Sec. 2 step 3: acceptance exp(-beta dE)).
 * beta >= 0, +inf allowed; NaN or negative -> EINVAL.  Builds the two
 * integer thresholds on the host. */
int ising_set_beta(ising_lattice *h, double beta);

/* The thresholds in use: host_thr[0] = thr for a = 0 (dE = 8),
 * host_thr[1] = thr for a = 1 (dE = 4); each in [0, 2^32]. */
int ising_get_thresholds(ising_lattice *h, uint64_t host_thr[2]);

/* Run n >= 0 full sweeps t+1 .. t+n (t += n).  A sweep is the paper's Monte
 * Carlo iteration (Sec. 2: every spin proposed once), in checkerboard order:
 * all colour-0 sites, then all colour-1 sites.  Asynchronous on the stream
 * (the first call on the on-chip path or with graph replays allocates its
 * mask buffer), except on the cluster path with several clusters, where the
 * call synchronises the stream to read the status of the waits between
 * clusters.  Errors: EINVAL (NULL, n < 0), ENOMEM (that buffer), ETIMEOUT
 * (a wait between clusters gave up; see ising_set_clusters), ECUDA. */
int ising_sweep(ising_lattice *h, int64_t n);

/* Run n sweeps and record E and M after sweeps t+every, t+2*every, ...:
 * host_E and host_M (caller-owned host arrays) receive n / every entries
 * each; either may be NULL.  n >= 0, 1 <= every <= 2^22.  Synchronises the stream.
 * The counts come from the reduction fused into the colour-1 half-sweep.
 * Errors: EINVAL (NULL, n < 0, every out of range), ENOMEM (the mask
 * buffer of the on-chip path or of the graph replays), ETIMEOUT (as for
 * ising_sweep), ECUDA. */
int ising_sweep_record(ising_lattice *h, int64_t n, int64_t every,
                       int64_t *host_E, int64_t *host_M);

/* Current energy (Eq. 1, Sec. 5.3) / magnetisation, exact.  Synchronises.
 * Errors: EINVAL (NULL), ECUDA. */
int ising_energy(ising_lattice *h, int64_t *host_E);
int ising_magnetization(ising_lattice *h, int64_t *host_M);

/* Eq. 2: the averages over n recorded sweeps of an L x L lattice, per spin:
 * *mean_e = (sum_t E_t) / (n L^2) and *mean_absm = (sum_t |M_t|) / (n L^2)
 * (the paper averages the per-iteration energies; the mean of |M_t| is the
 * magnetisation counterpart).  host_E and host_M are caller-owned host
 * arrays of n exact int64 records (as ising_sweep_record returns); either
 * may be NULL when its output is NULL.  The sums are exact (128-bit
 * integers) and each mean is one IEEE double division of the sum by n L^2,
 * so it is the correctly rounded quotient while |sum| and n L^2 are below
 * 2^53 (any run of fewer than about 2^21 records of the largest lattice).
 * Pure host arithmetic: no device work, no synchronisation.
 * Errors: EINVAL (n < 1, L invalid as for ising_create, an output whose
 * input array is NULL, both outputs NULL). */
int ising_means(const int64_t *host_E, const int64_t *host_M, int64_t n, int32_t L,
                double *mean_e, double *mean_absm);

/* Copy the spins to / from a caller-owned host array of n = L*L int8 values,
 * row-major s[i*L + j], each +1 or -1 (set: any value > 0 counts as +1).
 * Packing and unpacking run on the device through an int8 L*L staging
 * buffer that the library allocates on first use (also for ising_create_on
 * lattices) and frees in ising_destroy; ising_set_spins reads a pinned host
 * array (cudaHostAlloc / cudaHostRegister) in place instead, in one pass.
 * n != L*L -> EINVAL.  Synchronises.  Neither changes t. */
int ising_get_spins(ising_lattice *h, int8_t *host_out, size_t n);
int ising_set_spins(ising_lattice *h, const int8_t *host_in, size_t n);

/* Run a sequence of lattice states: for k = 0 .. nstates-1, ising_set_spins
 * with states[k] (L*L int8, row-major, > 0 is up), then ising_sweep_record of
 * `sweeps` sweeps with a record every `every`-th sweep, into E / M entries
 * k*R .. k*R + R - 1, R = sweeps / every (caller-owned host arrays of
 * nstates*R entries, either may be NULL).  The sweep counter continues
 * across states, so the results are those of the calls made one after
 * another.  The library copies state k + 1 to the device, on a copy stream
 * and into a second input buffer, while the sweeps of state k run.  With
 * pinned host arrays (cudaHostAlloc / cudaHostRegister) the copies overlap
 * the sweeps; pageable arrays work but do not overlap.  The arrays must stay
 * unchanged until the call returns.  On the on-chip path, with the
 * interleaved layout, or with more than 1024 records per state, the calls
 * run in turn.  No counterpart in the paper (input streaming).
 * Synchronises.  Errors: EINVAL (null state, sweeps > 2^30, every out of
 * 1..2^22), ENOMEM, ETIMEOUT (as for ising_sweep), ECUDA. */
int ising_run_states(ising_lattice *h, const int8_t *const *states, int32_t nstates, int64_t sweeps,
                     int64_t every, int64_t *E, int64_t *M);


/* The packed colour arrays, for checkpoints: n64 = 2 * L * pitch words,
 * colour 0 first, each colour row-major with `pitch` words per row (see
 * ising_layout).  Synchronises. */
int ising_get_words(ising_lattice *h, uint64_t *host_out, size_t n64);
int ising_set_words(ising_lattice *h, const uint64_t *host_in, size_t n64);

/* Layout facts: words per colour-row W, row pitch in words, live fields in
 * the last word of a row (1..21).  Any pointer may be NULL. */
int ising_layout(ising_lattice *h, int32_t *W, int32_t *pitch, int32_t *last_fields);

/* Sweep counter t (checkpoint / resume: with the counter-based draws a run
 * resumed at t is bit-identical to an uninterrupted one). */
int ising_get_sweep(ising_lattice *h, uint64_t *t);
int ising_set_sweep(ising_lattice *h, uint64_t t);

/* Use cudaStream_t `stream` (NULL = legacy default stream) from now on. */
int ising_set_stream(ising_lattice *h, void *stream);

/* Launch shape of the half-sweep kernels: rows_per_thread must be 4 (one
 * Philox call serves four rows).  block_words == 0 selects a 1-D grid over
 * the thread items (item = row group * W + word, no padding columns) with
 * block_groups threads per block, in {64, 128, 192, 256}.  Otherwise a 2-D
 * grid: block_words (threads along a row) in {16, 32, 64}; block_groups
 * (threads down the columns) in {1, 2, 4, 8, 16}; 32 <= block_words *
 * block_groups <= 256.  Default 4, 0, 128 (1-D, 128 threads).  Results do
 * not depend on the shape (the draws are keyed by site).  It shapes the
 * launches that draw inside the half-sweep: above 102400 thread items, and
 * the sweeps left over after the graph replays below that. */
int ising_set_tiling(ising_lattice *h, int32_t rows_per_thread,
                     int32_t block_words, int32_t block_groups);

/* Lanes per thread item on the launch path: 1, 2, 4 or 8, or 0 (default)
 * for the library's choice by lattice size (4 up to 8192 items, i.e. L up to
 * about 1100; 1 above).  With F lanes, lane q of an item
 * (4 rows x 1 word) draws the fields q, q + F, ... and the lanes merge their
 * accept bits with warp shuffles: F times the threads, each with 1/F of the
 * item's Philox calls.  This fills the GPU for lattices whose one thread
 * per item would leave SMs idle.  It applies to the launches that draw
 * inside the half-sweep (the sweeps left over after the graph replays,
 * whose half-sweeps apply masks drawn ahead).  No counterpart in the paper
 * (a scheduling choice); results do not depend on it.  Row-packed layout
 * only (EINVAL otherwise; EINVAL for other values). */
int ising_set_item_lanes(ising_lattice *h, int32_t lanes);

/* Execution path of ising_sweep / ising_sweep_record.  ISING_PATH_LAUNCHES:
 * two kernel launches per sweep, all SMs; up to 102400 thread items (L up
 * to about 4100, either layout) the launches of chunks of up to 32 sweeps are
 * captured once into CUDA graphs and replayed (recaptured after
 * ising_set_beta, ising_set_rng, ising_set_tiling, ising_set_item_lanes; a
 * device record index picks the count slots of each replay), because there
 * a half-sweep runs about as long as the host takes to launch it.  These
 * graphs draw the accept masks of up to 8 sweeps at a time on all SMs, into
 * two buffers the library allocates on first use (at most 33.5 MB), and
 * their half-sweeps only apply them.
 * ISING_PATH_RESIDENT: temporal
 * blocking with the whole lattice on chip -- one block copies both colour
 * arrays into shared memory and runs all requested sweeps there in one
 * launch (lattices with 2 L pitch 8 bytes <= 220 KB, i.e. L up to about
 * 740; larger -> EINVAL); it removes the per-sweep launch latency that
 * bounds small lattices.  Up to 512 thread items (ceil(L/4) * ceil(L/42),
 * L <= 292) the accept masks of the requested sweeps are first drawn by all
 * SMs into a device buffer the library allocates on first use (up to
 * 16 MB), and the on-chip block only applies them, one or two rows per
 * thread.
 * ISING_PATH_CLUSTER: temporal blocking on one thread-block cluster (16
 * blocks where the device runs such a cluster, else 8).  Row-packed
 * lattices with at least two rows per block whose window fits a block's
 * shared memory (L from 32 up to 1600): block b keeps rows b L / C ..
 * (b + 1) L / C - 1 of both colours in shared memory for a piece of up to
 * 256 sweeps.  Column-interleaved lattices (L from 84 up to 1512): block b
 * keeps a band of word columns (multiples of 4) of all N word rows.
 * Otherwise EINVAL, and EINVAL on a device without clusters.  After every
 * k <= 12 half-sweeps each block writes its first and last k own rows (or
 * columns) into its neighbours' shared memory (distributed shared memory)
 * and the blocks pass a cluster barrier; then they run k half-sweeps on
 * their own rows plus halo.  The accept masks of each
 * piece are drawn by the SMs the cluster leaves free, while the piece before
 * is applied, into two device buffers the library allocates on first use (up
 * to 256 MB together; 2 L pitch 8 bytes per sweep).  No spin-waits: only the
 * hardware's block and cluster barriers.
 * Both layouts may run several clusters per launch (see
 * ising_set_clusters), which takes the path past the sizes one cluster's
 * shared memory holds.
 * ISING_PATH_AUTO (default), row-packed: resident up to 128 thread items
 * (L <= 128), the cluster path above that up to L = 3000 (one cluster up to
 * L = 558, then 3 to 6 by size), the launch path above that (on a device
 * without clusters: resident up to 512 items, L <= 292, then the launch
 * path); column-interleaved: the cluster path up to L = 2604 (one cluster up
 * to L = 840, then 3 to 5), the launch path above.
 * Results are identical on every path. */
#define ISING_PATH_AUTO 0
#define ISING_PATH_LAUNCHES 1
#define ISING_PATH_RESIDENT 2
#define ISING_PATH_CLUSTER 3
int ising_set_path(ising_lattice *h, int32_t path);

/* The path the next ising_sweep / ising_sweep_record of the checkerboard
 * chain takes (ISING_PATH_RESIDENT, ISING_PATH_CLUSTER or
 * ISING_PATH_LAUNCHES; with the random-word chain, the path last set). */
int ising_get_path(ising_lattice *h, int32_t *path);

/* Clusters of one cluster-path launch: 0 = automatic
 * (the default), 1 .. 16 = that many thread-block clusters whose blocks own
 * consecutive row bands.  Inside a cluster the halo rows travel through
 * distributed shared memory; between clusters the two boundary blocks pass
 * them through a small device buffer the library allocates on first use
 * (clusters x 8 k pitch 8 bytes, k <= 12) with release/acquire flags.  A
 * flag wait gives up after one second of the GPU's clock.  A launch with
 * several clusters writes its lattice rows back only if all its blocks were
 * resident together, which all its blocks agree on at their end.  If they
 * were not (other work on the device held SMs, so waits gave up), the
 * launch writes nothing, the rest of the call runs on the launch path with
 * the same results, and the automatic choice keeps to one cluster until the
 * next ising_set_path or ising_set_clusters.  If a wait gave up while all
 * blocks were resident, the call returns ISING_ETIMEOUT, the sweeps it ran
 * are void, and the sweep counter has advanced (restore a checkpoint with
 * ising_set_words, or ising_set_spins in the column-interleaved layout, and
 * ising_set_sweep to retry).  A number of clusters the device cannot hold at
 * once, or for which the lattice has no window plan, gives EINVAL.
 * Column-interleaved lattices split their word columns the same way (k halo
 * columns of all word rows between clusters).  Results do not depend on it. */
int ising_set_clusters(ising_lattice *h, int32_t clusters);

/* Test hook of that wait: the next `launches` cluster-path launches with
 * several clusters wait for flag values no push reaches, so every wait
 * between clusters gives up after its second and the call returns
 * ISING_ETIMEOUT (the GPU keeps running; nothing traps).  0 clears it. */
int ising_cluster_inject_stall(ising_lattice *h, int32_t launches);

/* Test hook of that agreement: the launch with several clusters that comes
 * after `after` (>= 0) more such launches counts on one block more than it
 * has, so its blocks agree after 0.1 s that not all were resident and write
 * nothing; the call finishes on the launch path (results unchanged).  -1
 * clears it; below -1: EINVAL. */
int ising_cluster_inject_absent(ising_lattice *h, int32_t after);

/* Which Markov chain ising_sweep and ising_sweep_record run.
 * ISING_CHAIN_CHECKERBOARD (default): the checkerboard sweeps of the
 * conventions above (nstrips ignored).  ISING_CHAIN_RANDOM_WORDS: the paper's
 * own chain (Sec. 4 and 5, Appendix A), on a column-interleaved lattice only
 * (EINVAL otherwise): memory word (I, J) holds the spins (I + kN, J),
 * k = 0..20, N = L / 21; the L word columns form nstrips strips of
 * NC = L / nstrips >= 2 columns (the paper's processes; nstrips = 1 is its
 * one-process program); an iteration is phase 0, in which every strip
 * performs 10 N floor(NC/2) updates of words drawn uniformly with
 * replacement from its left floor(NC/2) columns, then phase 1 on its other
 * NC - floor(NC/2) columns.  An update applies the Metropolis rule to all 21
 * spins of its word at once.  Draws: update s of strip q in phase p of
 * iteration t takes the 24 words w[4b + e] of the Philox4x32-10 blocks
 * b = 0..5 with key (lo32(seed), hi32(seed)) and counter
 * (s, 8q + b, lo32(t), 2^31 | hi32(t) << 1 | p): row floor(w[0] N / 2^32),
 * column floor(w[1] h / 2^32) of the half strip's h columns, and w[2 + k]
 * for spin k (always 10 rounds, whatever ising_set_rng chose).  With this
 * chain the functions' "sweep" is the paper's iteration (10 update attempts
 * per spin on average, Table 2), and t counts iterations.  The strips of a
 * phase run in parallel, each strip's updates in its own sequence order, so
 * the result equals the sequential chain's.  Execution: the draws of an
 * iteration's updates are made first on all SMs, into a buffer of
 * 160 L^2 / 21 bytes the library allocates on first use (up to 256 MB,
 * L <= about 5900); with ISING_PATH_LAUNCHES, or above that size, each strip
 * draws its own updates.  A strip whose words fit in shared memory (N (h + 2)
 * words <= 160 KB) keeps them there for the phase.  Results are the same on
 * every form.  Errors: EINVAL (bad chain, nstrips not dividing L or
 * L / nstrips < 2, a row-packed lattice). */
#define ISING_CHAIN_CHECKERBOARD 0
#define ISING_CHAIN_RANDOM_WORDS 1
int ising_set_chain(ising_lattice *h, int32_t chain, int32_t nstrips);

/* Random-number scheme of the sweeps.  ISING_RNG_PHILOX4X32_10 (default) is
 * the generator of the conventions above.  ISING_RNG_PHILOX4X32_7 is an
 * opt-in cheaper member of the same family: the same keying and counters,
 * the iteration stopped after 7 rounds (Salmon et al. report 7 as the fewest
 * rounds at which Philox4x32 passed their test batteries; 10 keeps a safety
 * margin).  It gives a different, equally reproducible trajectory with the
 * same stationary distribution; the hot start always uses 10 rounds. */
#define ISING_RNG_PHILOX4X32_10 0
#define ISING_RNG_PHILOX4X32_7 1
int ising_set_rng(ising_lattice *h, int32_t scheme);

/* Device pointer to the colour-c array (c = 0 or 1), for zero-copy use by
 * other device code on the same stream.  Returned in *dev_ptr. */
int ising_device_words(ising_lattice *h, int32_t c, void **dev_ptr);

/* Fill host_out[4*n] with Philox4x32-10 blocks computed on the device:
 * block k = Philox(counter = host_ctr[4k .. 4k+3], key = (lo32(seed),
 * hi32(seed))).  Test hook for the generator every sweep uses.  Synchronises
 * the legacy default stream.  n <= 2^24. */
int ising_philox_blocks(uint64_t seed, const uint32_t *host_ctr, uint32_t *host_out,
                        int64_t n);


/* ---- Batches of independent replicas --------------------------------------
 * Many lattices of uneven size, each at its own temperature and seed, swept
 * together: every half-sweep of every replica runs in ONE kernel launch whose
 * blocks are tiles of the replicas (a tile table built at creation), and a
 * chunk of sweeps is captured once into a CUDA graph and replayed.  This
 * covers the paper's energy-versus-temperature scan (Sec. 5, one replica per
 * temperature).  Each replica's results are bit-identical to a single
 * ising_lattice with the same L, seed, beta and start: the draws are keyed by
 * (seed, sweep, colour, site) and do not depend on the tiling. */
typedef struct ising_batch ising_batch;   /* opaque, library-owned */

/* Create n >= 1 replicas.  Replica r: side L[r] (as ising_create), inverse
 * temperature beta[r] (as ising_set_beta), seed seed[r], hot start if
 * hot[r] != 0 (as ising_init_hot) else all +1, and t = 0.  All arrays are
 * caller-owned host arrays of n entries; hot may be NULL (all cold).  One
 * device allocation holds every replica.  The batch owns a non-blocking CUDA
 * stream (graph capture needs one).  Errors: EINVAL, ENOMEM, ECUDA. */
int ising_batch_create(int32_t n, const int32_t *L, const double *beta,
                       const uint64_t *seed, const uint8_t *hot, ising_batch **out);

int ising_batch_destroy(ising_batch *b);

/* Replica r runs sweeps[r] >= 0 sweeps (t_r+1 .. t_r+sweeps[r]); all
 * replicas advance in lockstep and a replica whose sweeps are done drops
 * out.  E and M are recorded after every `every`-th sweep of each replica:
 * host_E[r] / host_M[r] (caller-owned host arrays of sweeps[r] / every
 * entries; any of them, or host_E / host_M themselves, may be NULL).
 * Synchronises the batch's stream. */
int ising_batch_sweep(ising_batch *b, const int64_t *sweeps, int64_t every,
                      int64_t **host_E, int64_t **host_M);

/* Spins of replica r (as ising_get_spins, n = L[r]^2).  Synchronises. */
int ising_batch_get_spins(ising_batch *b, int32_t r, int8_t *host_out, size_t n);

/* Sweep counter of replica r. */
int ising_batch_get_sweep(ising_batch *b, int32_t r, uint64_t *t);

/* Random-number scheme of every replica (as ising_set_rng). */
int ising_batch_set_rng(ising_batch *b, int32_t scheme);

/* Threads per tile (64, 128 or 256; default 128) and sweeps per captured
 * graph (1 .. 1024; default 50).  Rebuilds the tile table.  Results do not
 * depend on either. */
int ising_batch_set_tiling(ising_batch *b, int32_t threads_per_tile, int32_t graph_chunk);

/* Lanes (1 .. 8; default 2): the replicas are split, largest first, into
 * `lanes` groups of about equal work (sum of L^2), and each group is an
 * independent branch of the captured graph, so the blocks of one lane can
 * fill SMs that another lane's last wave of blocks leaves idle.  No
 * counterpart in the paper (it is a scheduling choice).  Synchronises the
 * batch's stream and rebuilds the tile table.  Results do not depend on it.
 * Errors: EINVAL (lanes out of range), ENOMEM, ECUDA. */
int ising_batch_set_lanes(ising_batch *b, int32_t lanes);

/* One call (the batch entry of the C ABI): create, sweep, copy each
 * replica's final spins to final_spins[r] (host arrays of L[r]^2 int8; the
 * array or any entry may be NULL), destroy. */
int ising_batch_run(int32_t n, const int32_t *L, const double *beta, const uint64_t *seed,
                    const uint8_t *hot, const int64_t *sweeps, int64_t every,
                    int64_t **host_E, int64_t **host_M, int8_t **final_spins);

/* ---- Serving: continuous batching of simulation jobs -----------------------
 * The paper has no counterpart: it runs one lattice per MPI job.  A server owns a fixed device arena (its HBM budget) and a worker thread.
 * Jobs (L, beta, seed, start, sweeps) are admitted in arrival order while a
 * slot and arena space are free; every admitted job advances in epochs of
 * the batched half-sweep together with all other running jobs, so jobs that
 * arrive while others run join at the next epoch boundary.  A job's results
 * are bit-identical to running it alone (ising_lattice with the same
 * arguments): its draws depend only on its own seed and sweep numbers. */
typedef struct ising_server ising_server;   /* opaque, library-owned */

typedef struct ising_job {
    int32_t L;            /* lattice side, as ising_create */
    double beta;          /* inverse temperature, >= 0 */
    uint64_t seed;        /* Philox seed */
    int32_t hot;          /* != 0: hot start, else all +1 */
    int64_t sweeps;       /* >= 1 */
    int64_t every;        /* record E/M after sweeps every, 2*every, ... (>= 1) */
    int64_t *host_E;      /* caller-owned, sweeps / every entries, or NULL */
    int64_t *host_M;      /* caller-owned, sweeps / every entries, or NULL */
    int8_t *host_spins;   /* caller-owned, L*L final spins, or NULL */
    int32_t rng;          /* ISING_RNG_PHILOX4X32_10 (0) or ISING_RNG_PHILOX4X32_7 (1) */
} ising_job;               /* the host arrays must stay valid until the job is done */

typedef struct ising_result {
    int32_t status;       /* ISING_OK done; ISING_EBUSY queued or running; < 0 failed */
    int32_t state;        /* 0 queued, 1 running, 2 done, 3 failed, 4 cancelled */
    double submit_s;      /* seconds since server creation (steady clock) */
    double start_s;       /* admission time, or -1 */
    double done_s;        /* completion time, or -1 */
    int64_t sweeps_done;
} ising_result;

/* Create a server on the current device with an arena of hbm_budget_bytes
 * (allocated once; at least 256 bytes, rounded down to a multiple of 256), at
 * most ISING_SERVER_DEFAULT_MAX_JOBS (256) concurrently running jobs and epochs
 * of ISING_SERVER_DEFAULT_EPOCH_SWEEPS (50) sweeps.  *out receives the handle.
 * Errors: EINVAL (out NULL, budget < 256), ENOMEM, ECUDA. */
#define ISING_SERVER_DEFAULT_MAX_JOBS 256
#define ISING_SERVER_DEFAULT_EPOCH_SWEEPS 50
int ising_server_create(size_t hbm_budget_bytes, ising_server **out);

/* ising_server_create with the two scheduling limits chosen by the caller:
 * at most max_jobs concurrently running jobs (1..4096) and epochs of
 * epoch_sweeps sweeps (1..100000), max_jobs * epoch_sweeps <= 2^22 (the
 * device record buffer of one epoch).  Results do not depend on either.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int ising_server_create_ex(size_t hbm_budget_bytes, int32_t max_jobs, int32_t epoch_sweeps,
                           ising_server **out);

/* Queue a job (copied); *id receives its id.  Thread-safe.  Errors: EINVAL
 * (bad job), ENOMEM (the job alone exceeds the whole arena). */
int ising_server_submit(ising_server *srv, const ising_job *job, uint64_t *id);

/* Non-blocking status of job `id`.  Thread-safe.  ENOTFOUND for an unknown
 * (or already released) id. */
int ising_server_poll(ising_server *srv, uint64_t id, ising_result *out);

/* Wait up to timeout_ms (< 0: forever) for job `id` to finish; *out as poll.
 * Returns ISING_ETIMEOUT if it is still queued or running. */
int ising_server_wait(ising_server *srv, uint64_t id, int64_t timeout_ms, ising_result *out);

/* Cancel a job that is still queued (running jobs finish). */
int ising_server_cancel(ising_server *srv, uint64_t id);

/* Forget a finished job's record (its id becomes unknown). */
int ising_server_release(ising_server *srv, uint64_t id);

/* Totals since creation: jobs done, spin updates done, epochs run, seconds
 * the worker spent with at least one job on the device; any may be NULL. */
int ising_server_stats(ising_server *srv, int64_t *jobs_done, double *spin_updates, int64_t *epochs,
                       double *busy_s);

/* Stop the worker after the running jobs' current epoch, fail the queued
 * ones (state cancelled), free the arena.  Jobs still running are failed. */
int ising_server_destroy(ising_server *srv);

/* Failure-injection hook for tests (no counterpart in the paper): after
 * `epochs` more epochs (0: the next one), the worker throws a host exception
 * at the start of an epoch, before that epoch's device work.  The worker
 * catches it, waits for its streams, marks every running job failed with
 * status ISING_EINTERNAL, returns their arena blocks and goes on admitting
 * and running the queued jobs.  epochs = -1 disarms the hook.  Nothing
 * touches the device: no kernel is made to fault or hang.  Thread-safe.
 * Errors: EINVAL (NULL, epochs < -1). */
int ising_server_inject_fault(ising_server *srv, int32_t epochs);

/* ---- Autotuning ---------------------------------------------------------
 * No counterpart in the paper.  Time the candidate launch shapes on the current device and return the
 * fastest.  Every candidate must leave a bit-identical lattice (the draws are
 * keyed by site, not by thread); a difference returns ISING_ECUDA.  The
 * caller applies the choice (ising_set_tiling / ising_set_path,
 * ising_batch_set_tiling); the Python binding keeps the choices in a JSON
 * table. */

/* Single lattice of side L: the launch shapes of ising_set_tiling (1-D with
 * 64/128/192/256 threads, eleven 2-D block_words x block_groups) with one
 * thread per item, the 1-D shape with 2, 4 and 8 lanes per item
 * (ising_set_item_lanes) and, if the lattice fits, the on-chip path;
 * `sweeps` timed sweeps each (1..100000) from a hot start at T = 2.269.
 * best_item_lanes is 0 for the on-chip path.  Outputs may be NULL. */
int ising_autotune(int32_t L, int32_t sweeps, int32_t *best_block_words, int32_t *best_block_groups,
                   int32_t *best_path, int32_t *best_item_lanes, double *ns_per_update);

/* Batch (arguments as ising_batch_create): threads per tile {64, 128, 256}
 * x graph chunk {10, 50, 200} x lanes {1, 2, 4}, `sweeps` timed sweeps per
 * replica with E/M every `every`-th sweep (1 <= every <= sweeps; the
 * kernels differ for every == 1).  Outputs may be NULL. */
int ising_batch_autotune(int32_t n, const int32_t *L, const double *beta, const uint64_t *seed,
                         const uint8_t *hot, int64_t sweeps, int64_t every, int32_t *best_threads,
                         int32_t *best_chunk, int32_t *best_lanes, double *ns_per_update);

/* Throughput probe of the integer instructions the sweep is made of, for the
 * roofline (no counterpart in the paper): on the current device, one block
 * of 1024 threads per SM runs 8 independent dependency chains per thread of
 * (a) 32x32 -> 64-bit products as a Philox round forms them (both halves,
 * folded back by an XOR on the other pipe), (b) 32-bit multiply-adds and
 * (c) three-input logic ops, timed with the SM's cycle counter.  Outputs (any may be NULL): lane operations per SM per clock
 * of each kind (the median over the SMs), and the SM count.  Takes a few
 * milliseconds; allocates and frees about 0.6 MB of device memory and
 * synchronises the device.  Errors: ENOMEM, ECUDA. */
int ising_probe_int_pipes(double *mulwide_per_sm_clk, double *mad32_per_sm_clk, double *lop3_per_sm_clk,
                          int32_t *sm_count);

/* Memory-safety check of the checked build (no counterpart in the paper).  A
 * library built with -DISING_CHECKED (paper_1811_04384_gb300.build.build(
 * checked=True), libising_checked.so) range-checks every lattice-word index of
 * the sweep, apply, batch, on-chip, column-interleaved and random-word
 * kernels against the array it indexes; an index out of range is not
 * accessed (loads give 0, stores are dropped, nothing traps) and the first
 * one is recorded on the device.  *checked = 1 for that build, 0 for the
 * normal one (whose kernels check nothing).  *first_violation = 0 if no index
 * was out of range since the previous call, else bit 63 set, the source line
 * of the access in bits 40..62 and the low 40 bits of the index; the call
 * clears the record.  Synchronises the device.  Either output may be NULL.
 * Errors: ECUDA. */
int ising_check_status(int32_t *checked, uint64_t *first_violation);

/* ---- Allocation-free record path ----------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: for example a plug-in running inside a host program
 * that owns all device memory through its own pool, or a latency-critical
 * loop in which an allocation (which may synchronise the device) is not
 * acceptable.  It runs the same sweeps and fused energy/magnetisation
 * reduction as ising_sweep_record, but on a packed lattice the caller owns,
 * and it allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * dev_words0 / dev_words1: caller-owned device arrays of colour 0 and 1 in
 * the library's packed layout (L rows x pitch words each, as ising_layout()
 * and ising_device_words() describe), updated in place.  Sweeps t0+1 ..
 * t0+n run with key `seed` at inverse temperature `beta`; host_E and host_M
 * (caller-owned host arrays, either may be NULL) receive the n / every
 * records taken after sweeps t0+every, t0+2*every, ...  No handle and no
 * sweep counter is involved: the caller tracks t.  Work is ordered on
 * cudaStream_t `stream` (NULL = legacy default stream); the call
 * synchronises it before returning.
 *
 * Scratch: the count slots, per-record results and sweep counter live in one
 * fixed file-scope device array of about 528 KB, which every GPU that loads
 * the library holds until the process exits.  It holds at most
 * ISING_NOALLOC_MAX_RECORDS records per call; n / every above that returns
 * ISING_EINVAL before any device work.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  That address
 * is cached per device for the life of the process: after cudaDeviceReset
 * (or a reset of the device's primary context) the cached address is stale,
 * so do not call this entry point on that device again in the same process.
 * Every call shares the array, which keeps the previous call's contents
 * (each call clears the slots it uses first): calls that overlap on the GPU,
 * on any streams, race and give wrong results.
 *
 * Execution: two plain half-sweep launches per sweep with a fixed 2-D shape
 * (32 words x 4 row groups per block), no CUDA graphs and no on-chip path,
 * so small lattices run at the plain-launch rate, far below
 * ising_sweep_record's; results are identical (the draws are keyed by site).
 * Errors: EINVAL (NULL words, bad L, n < 0, every < 1, beta < 0 or NaN, too
 * many records), ECUDA. */
#define ISING_NOALLOC_MAX_RECORDS 1024
int ising_sweep_record_noalloc(uint64_t *dev_words0, uint64_t *dev_words1, int32_t L,
                               uint64_t seed, double beta, uint64_t t0, int64_t n,
                               int64_t every, int64_t *host_E, int64_t *host_M,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */

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
    ISING_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    ISING_EBUSY = -5,     /* no free slot / budget (server admission) */
    ISING_ENOTFOUND = -6  /* unknown request id */
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

/* Release the handle and every device buffer the library allocated for it
 * (not a caller-owned dev_buf).  NULL is accepted. */
int ising_destroy(ising_lattice *h);

/* Hot start (Sec. 5.1: every spin up or down at random): s(i,j) = +1 iff the
 * site's Philox draw at t = 0 is below 2^31.  Resets t to 0. */
int ising_init_hot(ising_lattice *h);

/* Cold start: every spin = `spin` (+1 or -1, else EINVAL).  Resets t to 0. */
int ising_init_cold(ising_lattice *h, int8_t spin);

/* Set the inverse temperature (Sec. 2 step 3: acceptance exp(-beta dE)).
 * beta >= 0, +inf allowed; NaN or negative -> EINVAL.  Builds the two
 * integer thresholds on the host. */
int ising_set_beta(ising_lattice *h, double beta);

/* The thresholds in use: host_thr[0] = thr for a = 0 (dE = 8),
 * host_thr[1] = thr for a = 1 (dE = 4); each in [0, 2^32]. */
int ising_get_thresholds(ising_lattice *h, uint64_t host_thr[2]);

/* Run n >= 0 full sweeps t+1 .. t+n (t += n).  Asynchronous on the stream. */
int ising_sweep(ising_lattice *h, int64_t n);

/* Run n sweeps and record E and M after sweeps t+every, t+2*every, ...:
 * host_E and host_M (caller-owned host arrays) receive n / every entries
 * each; either may be NULL.  n >= 0, every >= 1.  Synchronises the stream.
 * The counts come from the reduction fused into the colour-1 half-sweep. */
int ising_sweep_record(ising_lattice *h, int64_t n, int64_t every,
                       int64_t *host_E, int64_t *host_M);

/* Current energy (Eq. 1, Sec. 5.3) / magnetisation, exact.  Synchronises. */
int ising_energy(ising_lattice *h, int64_t *host_E);
int ising_magnetization(ising_lattice *h, int64_t *host_M);

/* Copy the spins to / from a caller-owned host array of n = L*L int8 values,
 * row-major s[i*L + j], each +1 or -1 (set: any value > 0 counts as +1).
 * Packing and unpacking run on the device.  n != L*L -> EINVAL.
 * Synchronises.  Neither changes t. */
int ising_get_spins(ising_lattice *h, int8_t *host_out, size_t n);
int ising_set_spins(ising_lattice *h, const int8_t *host_in, size_t n);

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

/* Launch shape of the half-sweep kernels: rows_per_thread in {4, 8},
 * block_words (threads along a row) in {16, 32, 64}, block_groups (threads
 * along the columns) in {1, 2, 4, 8, 16}; block_words * block_groups <= 512.
 * Results do not depend on the shape (the draws are keyed by site). */
int ising_set_tiling(ising_lattice *h, int32_t rows_per_thread,
                     int32_t block_words, int32_t block_groups);

/* Device pointer to the colour-c array (c = 0 or 1), for zero-copy use by
 * other device code on the same stream.  Returned in *dev_ptr. */
int ising_device_words(ising_lattice *h, int32_t c, void **dev_ptr);

/* Fill host_out[4*n] with Philox4x32-10 blocks computed on the device:
 * block k = Philox(counter = host_ctr[4k .. 4k+3], key = (lo32(seed),
 * hi32(seed))).  Test hook for the generator every sweep uses.  Synchronises
 * the legacy default stream.  n <= 2^24. */
int ising_philox_blocks(uint64_t seed, const uint32_t *host_ctr, uint32_t *host_out,
                        int64_t n);


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
 * current; make that first call before any stream capture.  Every call
 * shares the array, which keeps the previous call's contents (each call
 * clears the slots it uses first): calls that overlap on the GPU, on any
 * streams, race and give wrong results.
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

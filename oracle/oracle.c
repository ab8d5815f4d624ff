/*
 * Oracle: a plain, slow, single-threaded CPU model of the multi-spin Ising
 * Metropolis chain.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it; the product library never does.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * One int8 per spin (+1 / -1), row-major s[i*L + j], i = row, j = column.
 *
 * What it follows (Hassani & Rafibakhsh, "Parallelization and implementation
 * of multi-spin Monte Carlo simulation of 2D square Ising model using MPI and
 * C++"):
 *   - Eq. 1, Sec. 2: H = -J sum_<mn> s_m s_n over nearest neighbours, periodic
 *     boundary conditions, J = 1, K = 1, no field.
 *   - Sec. 2, steps 1-3: a proposed flip with dE <= 0 is accepted; otherwise it
 *     is accepted with probability exp(-dE/KT).
 *   - Eq. 3 and Table 1: the per-spin "group value" a is the number of the four
 *     nearest neighbours anti-aligned with the spin, and dE = 8J - 4Ja.
 *   - Sec. 5.3: the energy is the sum over right and down bonds.
 *   - Eq. 2: averages are taken over the per-iteration energies.
 *
 * Readings where the paper is silent (all stated in the design notes):
 *   - Visit order: checkerboard.  Sweep t updates colour 0 ((i+j) even) for
 *     every site, then colour 1.  Same-colour sites are never neighbours, so an
 *     in-place loop equals a simultaneous update of the colour.
 *   - Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *     (lo32(seed), hi32(seed)), counter = (i>>2, j>>1, lo32(t), hi32(t)<<1 | c),
 *     the site's draw r is output word (i & 3).
 *   - Acceptance: a >= 2 always flips; a in {0,1} flips iff r < thr[a], with
 *     thr[0] = floor(2^32 exp(-8 beta)), thr[1] = floor(2^32 exp(-4 beta)),
 *     evaluated in IEEE double.
 *   - Hot start (t = 0): s = +1 iff the site's Philox draw at t = 0 is < 2^31.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox (SC'11, Sec. 3): a Feistel-like bijection of the counter, keyed by
 * k, with round function  (x0,x1,x2,x3) -> (hi(M1*x2)^x1^k0, lo(M1*x2),
 * hi(M0*x0)^x3^k1, lo(M0*x0))  and the key bumped by the Weyl constants
 * between rounds.  Written twice, for 32-bit and 64-bit words, with the same
 * structure, so that the 64-bit member can be checked against an independent
 * published implementation. */

/* Philox4x32 with `rounds` rounds (SC'11 defines the family; 10 is its
 * recommended member, 7 the fewest rounds at which its authors found it to
 * pass their statistical test batteries). */
void ora_philox4x32_r(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < rounds; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    ora_philox4x32_r(ctr, key, 10, out);
}

void ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Number of Philox rounds the sweeps use: 10 (default) or 7 (an opt-in
 * cheaper scheme).  The hot start always uses 10. */
static int g_sweep_rounds = 10;

void ora_set_sweep_rounds(int rounds) { g_sweep_rounds = rounds; }

/* The uint32 draw of site (i, j) at sweep t with `rounds` Philox rounds. */
uint32_t ora_site_draw_r(uint64_t seed, uint64_t t, int i, int j, int rounds)
{
    int c = (i + j) & 1;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)(i >> 2), (uint32_t)(j >> 1),
                        (uint32_t)t, ((uint32_t)(t >> 32) << 1) | (uint32_t)c };
    uint32_t out[4];
    ora_philox4x32_r(ctr, key, rounds, out);
    return out[i & 3];
}

/* The uint32 draw of site (i, j) at sweep t (t = 0: initialisation). */
uint32_t ora_site_draw(uint64_t seed, uint64_t t, int i, int j)
{
    return ora_site_draw_r(seed, t, i, j, 10);
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds.  Sec. 2 step 3: an uphill flip (dE > 0) is accepted
 * with probability exp(-dE/KT) = exp(-beta dE).  Table 1: a = 0 gives dE = 8J,
 * a = 1 gives dE = 4J.  The integer threshold makes P(r < thr) for a uniform
 * 32-bit r equal to floor(2^32 p) / 2^32. */
void ora_thresholds(double beta, uint64_t thr[2])
{
    const double two32 = 4294967296.0;
    for (int a = 0; a < 2; ++a) {
        double dE = 8.0 - 4.0 * (double)a;   /* J = 1 */
        double p = exp(-dE * beta);
        double x = floor(p * two32);
        if (x > two32) x = two32;
        if (x < 0.0) x = 0.0;
        thr[a] = (uint64_t)x;
    }
}

/* ------------------------------------------------------------------------ */
/* Local quantities (Eq. 3 and Table 1). */

static int wrap(int x, int L) { return ((x % L) + L) % L; }

/* a = number of the four nearest neighbours whose spin differs from s(i,j). */
int ora_group_value(int L, const int8_t *s, int i, int j)
{
    int8_t me = s[i * L + j];
    int8_t nb[4] = {
        s[wrap(i - 1, L) * L + j], s[wrap(i + 1, L) * L + j],
        s[i * L + wrap(j - 1, L)], s[i * L + wrap(j + 1, L)] };
    int a = 0;
    for (int n = 0; n < 4; ++n)
        if (nb[n] != me) ++a;
    return a;
}

/* dE of flipping s(i,j): E' - E with E = -J s sum(neighbours) (Table 1). */
int ora_delta_energy(int L, const int8_t *s, int i, int j)
{
    int8_t me = s[i * L + j];
    int sum = s[wrap(i - 1, L) * L + j] + s[wrap(i + 1, L) * L + j]
            + s[i * L + wrap(j - 1, L)] + s[i * L + wrap(j + 1, L)];
    int e_before = -me * sum;
    int e_after = me * sum;
    return e_after - e_before;
}

/* ------------------------------------------------------------------------ */
/* Observables.  Sec. 5.3: every bond is counted once as a right or down bond
 * of one site. */

int64_t ora_energy(int L, const int8_t *s)
{
    int64_t E = 0;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            int me = s[i * L + j];
            int right = s[i * L + wrap(j + 1, L)];
            int down = s[wrap(i + 1, L) * L + j];
            E -= (int64_t)me * right;
            E -= (int64_t)me * down;
        }
    return E;
}

int64_t ora_magnetization(int L, const int8_t *s)
{
    int64_t M = 0;
    for (size_t n = 0; n < (size_t)L * (size_t)L; ++n)
        M += s[n];
    return M;
}

/* ------------------------------------------------------------------------ */
/* Initialisation (Sec. 5.1: each spin drawn up or down at random). */

void ora_init_hot(int L, uint64_t seed, int8_t *s)
{
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            uint32_t r = ora_site_draw(seed, 0, i, j);
            s[i * L + j] = (r < 0x80000000u) ? (int8_t)1 : (int8_t)-1;
        }
}

void ora_init_cold(int L, int8_t v, int8_t *s)
{
    memset(s, 0, (size_t)L * (size_t)L);
    for (size_t n = 0; n < (size_t)L * (size_t)L; ++n)
        s[n] = v;
}

/* ------------------------------------------------------------------------ */
/* The Metropolis update of one colour at sweep t.
 * stats (may be NULL): 10 counters, [0..4] proposals with group value a,
 * [5..9] accepted flips with group value a. */
void ora_half_sweep(int L, int8_t *s, uint64_t seed, uint64_t t, int c,
                    const uint64_t thr[2], int64_t *stats)
{
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            if (((i + j) & 1) != c)
                continue;
            int a = ora_group_value(L, s, i, j);
            int flip;
            if (a >= 2) {
                flip = 1;                               /* dE <= 0 */
            } else {
                uint32_t r = ora_site_draw_r(seed, t, i, j, g_sweep_rounds);
                flip = ((uint64_t)r < thr[a]);          /* strict < */
            }
            if (stats) {
                stats[a] += 1;
                stats[5 + a] += flip;
            }
            if (flip)
                s[i * L + j] = (int8_t)(-s[i * L + j]);
        }
}

/* The same update restricted to rows i0 .. i1-1 (a strip of a row-strip
 * partition, Sec. 4): it reads rows i0-1 and i1 as halo rows. */
void ora_half_sweep_rows(int L, int8_t *s, uint64_t seed, uint64_t t, int c,
                         const uint64_t thr[2], int i0, int i1)
{
    for (int i = i0; i < i1; ++i)
        for (int j = 0; j < L; ++j) {
            if (((i + j) & 1) != c)
                continue;
            int a = ora_group_value(L, s, i, j);
            int flip = 1;
            if (a < 2) {
                uint32_t r = ora_site_draw_r(seed, t, i, j, g_sweep_rounds);
                flip = ((uint64_t)r < thr[a]);
            }
            if (flip)
                s[i * L + j] = (int8_t)(-s[i * L + j]);
        }
}

/* Many Philox4x32-10 blocks: out[4k..4k+3] = Philox(ctr[4k..4k+3], key). */
void ora_philox4x32_10_many(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t k = 0; k < n; ++k)
        ora_philox4x32_10(ctr + 4 * k, key, out + 4 * k);
}

void ora_sweep(int L, int8_t *s, uint64_t seed, uint64_t t, double beta, int64_t *stats)
{
    uint64_t thr[2];
    ora_thresholds(beta, thr);
    ora_half_sweep(L, s, seed, t, 0, thr, stats);
    ora_half_sweep(L, s, seed, t, 1, thr, stats);
}

/* Run sweeps t0+1 .. t0+n and record E, M after every `every`-th one, i.e.
 * after sweeps t0+every, t0+2*every, ...  (n / every entries). */
void ora_run(int L, int8_t *s, uint64_t seed, double beta, uint64_t t0,
             int64_t n, int64_t every, int64_t *E, int64_t *M)
{
    int64_t k = 0;
    for (int64_t step = 1; step <= n; ++step) {
        ora_sweep(L, s, seed, t0 + (uint64_t)step, beta, NULL);
        if (every > 0 && step % every == 0) {
            E[k] = ora_energy(L, s);
            M[k] = ora_magnetization(L, s);
            ++k;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The paper's own chain: random memory words (Sec. 4 and 5, Appendix A).
 *
 * The lattice is L x L with L = F N: the paper packs F = 21 spins into a
 * memory word and has N word rows.  Memory word (I, J), 0 <= I < N,
 * 0 <= J < L, holds the spins (I + kN, J), k = 0 .. F-1 (Sec. 3).  With
 * N >= 2 none of them neighbours another (their rows differ by multiples of
 * N, and the wrap from I + (F-1)N to I is N rows), so one word update can
 * decide all F spins from the configuration before it, as the paper's
 * `update` does.
 *
 * One Monte Carlo iteration t: the L word columns are split into nstrips
 * strips of NC = L / nstrips columns (the paper's processes, Sec. 4);
 * phase 0 updates the left floor(NC/2) columns of every strip, phase 1 the
 * remaining ones (Sec. 5.2).  In phase p a strip performs 10 N h_p word
 * updates, h_p being its number of columns in that phase (the paper's
 * noOfUpdatesP1 / noOfUpdatesP2: ten times the words of the half), each on
 * a word drawn uniformly with replacement from the half strip: a row from
 * 0 .. N-1 and a column from the h_p columns (Appendix A's row and column
 * generators).  A word update applies the Metropolis rule of Sec. 2 to each
 * of its spins: with a the number of anti-aligned neighbours (Eq. 3,
 * Table 1), a >= 2 flips, a in {0, 1} flips iff the spin's draw is below
 * thr[a].  The strips of one phase never update neighbouring words (a half
 * strip's neighbour columns belong to the other phase), so the order in
 * which they run does not change the result; the oracle runs them in order
 * 0, 1, ... (reverse != 0: in the opposite order, to test that claim).
 *
 * Draws (a reading: the paper reseeds ranlux48 from random_device, so its
 * runs cannot be replayed): update s of strip q in phase p of iteration t
 * takes the 24 words w[4b + e] of the Philox4x32-10 blocks b = 0 .. 5 with
 * key (lo32(seed), hi32(seed)) and counter
 * (s, 8q + b, lo32(t), 2^31 | hi32(t) << 1 | p).  Row I = floor(w[0] N / 2^32),
 * column = the half strip's first column + floor(w[1] h_p / 2^32), and spin
 * k of the word uses w[2 + k].  (The top counter bit keeps these draws apart
 * from the checkerboard chain's for every t < 2^62.)
 *
 * stats (may be NULL): int64[10], [0..4] proposals by a, [5..9] flips by a. */

static void rw_draws(uint64_t seed, uint64_t t, int phase, int strip, uint32_t step, uint32_t w[24])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int b = 0; b < 6; ++b) {
        uint32_t ctr[4] = { step, (uint32_t)strip * 8u + (uint32_t)b, (uint32_t)t,
                            0x80000000u | ((uint32_t)(t >> 32) << 1) | (uint32_t)phase };
        ora_philox4x32_10(ctr, key, w + 4 * b);
    }
}

/* The word a draw selects: row and column of the half strip [col0, col0 + h). */
void ora_rw_select(uint64_t seed, uint64_t t, int phase, int strip, uint32_t step, int N, int col0, int h,
                   int *I, int *J)
{
    uint32_t w[24];
    rw_draws(seed, t, phase, strip, step, w);
    *I = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
    *J = col0 + (int)(((uint64_t)w[1] * (uint64_t)h) >> 32);
}

/* One word update: spins (I + kN, J), k = 0 .. F-1, decided together. */
static void rw_update_word(int L, int F, int8_t *s, int I, int J, const uint32_t w[24],
                           const uint64_t thr[2], int64_t *stats)
{
    const int N = L / F;
    int flip[22];
    for (int k = 0; k < F; ++k) {
        int i = I + k * N;
        int a = ora_group_value(L, s, i, J);
        if (a >= 2) flip[k] = 1;
        else flip[k] = ((uint64_t)w[2 + k] < thr[a]);
        if (stats) {
            stats[a] += 1;
            stats[5 + a] += flip[k];
        }
    }
    for (int k = 0; k < F; ++k)
        if (flip[k]) s[(I + k * N) * L + J] = (int8_t)(-s[(I + k * N) * L + J]);
}

/* Update `step` of strip q in phase p of iteration t: choose the word in the
 * half strip [col0, col0 + h), then update it. */
void ora_rw_step(int L, int F, int8_t *s, uint64_t seed, uint64_t t, int phase, int q, uint32_t step,
                 int col0, int h, const uint64_t thr[2], int64_t *stats)
{
    const int N = L / F;
    uint32_t w[24];
    rw_draws(seed, t, phase, q, step, w);
    const int I = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
    const int J = col0 + (int)(((uint64_t)w[1] * (uint64_t)h) >> 32);
    rw_update_word(L, F, s, I, J, w, thr, stats);
}

void ora_rw_iteration(int L, int F, int8_t *s, uint64_t seed, uint64_t t, int nstrips,
                      const uint64_t thr[2], int reverse, int64_t *stats)
{
    const int N = L / F;
    const int NC = L / nstrips;
    for (int phase = 0; phase < 2; ++phase) {
        const int h = phase == 0 ? NC / 2 : NC - NC / 2;
        const uint32_t updates = 10u * (uint32_t)N * (uint32_t)h;
        for (int n = 0; n < nstrips; ++n) {
            const int q = reverse ? nstrips - 1 - n : n;
            const int col0 = q * NC + (phase == 0 ? 0 : NC / 2);
            for (uint32_t step = 0; step < updates; ++step)
                ora_rw_step(L, F, s, seed, t, phase, q, step, col0, h, thr, stats);
        }
    }
}

/* Iterations t0+1 .. t0+n at inverse temperature beta; E, M after every
 * `every`-th iteration (n / every entries), as ora_run does for sweeps. */
void ora_rw_run(int L, int F, int8_t *s, uint64_t seed, double beta, uint64_t t0, int64_t n,
                int64_t every, int nstrips, int64_t *E, int64_t *M, int64_t *stats)
{
    uint64_t thr[2];
    ora_thresholds(beta, thr);
    int64_t k = 0;
    for (int64_t it = 1; it <= n; ++it) {
        ora_rw_iteration(L, F, s, seed, t0 + (uint64_t)it, nstrips, thr, 0, stats);
        if (every > 0 && it % every == 0) {
            E[k] = ora_energy(L, s);
            M[k] = ora_magnetization(L, s);
            ++k;
        }
    }
}

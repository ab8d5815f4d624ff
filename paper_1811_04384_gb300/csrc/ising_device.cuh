// Device code of the multi-spin Ising Metropolis path (sm_103a).
//
// Layout (multi-spin coding of Sec. 3, 3-bit fields, 000 = down, 001 = up, 21
// spins per 64-bit word, bit 63 zero).  The paper interleaves 21 rows of one
// column into a word and needs L = 21N; here the spins of one colour in one
// row are packed along the row, so any even L works:
//   colour c = (i + j) & 1, m = j >> 1 in [0, L/2) indexes the colour-c sites
//   of row i; word w of colour-row (c, i) holds m = 21 w + k in field k
//   (bits 3k .. 3k+2); the last word of a row holds `rlast` live fields and
//   its dead fields stay zero.  Array c is row-major, `P` words per row.
//
// Neighbours of a colour-c site (i, m): up/down are field m of the
// other-colour rows i-1 / i+1; left/right are fields m and m-1 of row i when
// (i + c) is even, fields m and m+1 when it is odd (periodic in m over L/2).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "philox.cuh"

#ifndef ISING_INSERTS_ON_ALU
#define ISING_INSERTS_ON_ALU 0
#endif

namespace ising {

constexpr int kFields = 21;
constexpr uint64_t kSpinBits = 0x1249249249249249ull;   // bit 3k, k = 0..20
constexpr int kCountSlots = 32;                          // spread of the E/M atomics

struct Geom {
    int L;          // lattice side (even, >= 4)
    int W;          // words per colour-row = ceil((L/2) / 21)
    int P;          // row pitch in words (W rounded up to even)
    int rlast;      // live fields in the last word of a row (1..21)
};

// Per-launch constants of one half-sweep.
struct SweepArgs {
    const uint64_t* t_base;    // device: sweep counter before this chunk
    uint32_t t_off;            // this half-sweep belongs to sweep *t_base + t_off
    uint32_t thr0, thr1;       // integer thresholds clamped to 2^32 - 1 ...
    uint32_t all0, all1;       // ... and ~0u where the threshold is 2^32
    uint32_t one;              // the value 1, as a launch operand (see accept_insert)
    uint32_t rounds;           // Philox rounds of the sweep draws: 10 (default) or 7 (opt-in)
    PhiloxKeys rk;             // round keys of the key (lo32(seed), hi32(seed))
    unsigned long long* counts;  // E/M count slots of this record (RECORD only)
    const uint32_t* rec_base;    // device record index added to `counts` (graph replays), or null
};

// The 32 count slots a RECORD launch adds to: `counts`, moved on by
// *rec_base records when a replayed graph picks its slot on the device.
__device__ __forceinline__ unsigned long long* record_counts(const SweepArgs& a)
{
    return a.rec_base ? a.counts + (size_t)(*a.rec_base) * 2 * kCountSlots : a.counts;
}

// Programmatic dependent launch: a half-sweep launched with programmatic
// stream serialization lets the next half-sweep be launched and its blocks be
// placed as soon as every block of this one has started (launch_dependents),
// and waits, before its first read, until the previous grid has completed
// and its writes are visible (wait).  Both are no-ops in a plain launch.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- Checked build (compiled with -DISING_CHECKED) -------------------------
// Every lattice-word access of the sweep routines goes through word_ld /
// word_st with the length of the array it indexes.  In a checked build an
// index at or past that length is not accessed (a load gives 0, a store is
// dropped) and the first such index is recorded, with the source line of the
// access, in this translation unit's device word g_check_word; the host reads
// and clears the words of every translation unit (ising_check_status).
// Nothing traps or asserts, so a bad index leaves the context usable.  In the
// normal build these are plain accesses.
#ifdef ISING_CHECKED
static __device__ unsigned long long g_check_word;

__device__ __forceinline__ bool check_index(uint64_t idx, uint64_t n, uint32_t line)
{
    if (idx < n) return true;
    atomicCAS(&g_check_word, 0ull, (1ull << 63) | ((uint64_t)(line & 0x7FFFFFu) << 40) | (idx & 0xFFFFFFFFFFull));
    return false;
}

// Host side: this translation unit's word, read and cleared (registered with
// the library's list of readers when the library loads).
bool register_check_reader(int (*reader)(unsigned long long*));
static int read_check_word(unsigned long long* out)
{
    const unsigned long long zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_check_word, sizeof(zero));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(zero));
    return e == cudaSuccess ? 0 : -1;
}
static const bool g_check_reader_registered = register_check_reader(&read_check_word);
#endif

// A lattice word p[idx] of an array of n words: through the read-only cache
// (LDG) or a plain load.
template <bool LDG>
__device__ __forceinline__ uint64_t word_ld(const uint64_t* p, uint64_t idx, uint64_t n, uint32_t line)
{
#ifdef ISING_CHECKED
    if (!check_index(idx, n, line)) return 0;
#endif
    return LDG ? __ldg(p + idx) : p[idx];
}

__device__ __forceinline__ void word_st(uint64_t* p, uint64_t idx, uint64_t v, uint64_t n, uint32_t line)
{
#ifdef ISING_CHECKED
    if (!check_index(idx, n, line)) return;
#endif
    p[idx] = v;
}

__device__ __forceinline__ uint32_t half_ld(const uint32_t* p, uint64_t idx, uint64_t n, uint32_t line)
{
#ifdef ISING_CHECKED
    if (!check_index(idx, n, line)) return 0;
#endif
    return p[idx];
}

__device__ __forceinline__ void half_st(uint32_t* p, uint64_t idx, uint32_t v, uint64_t n, uint32_t line)
{
#ifdef ISING_CHECKED
    if (!check_index(idx, n, line)) return;
#endif
    p[idx] = v;
}

__device__ __forceinline__ uint64_t lattice_words(const Geom& g) { return (uint64_t)g.L * (uint64_t)g.P; }

__device__ __forceinline__ int wrap_row(int i, int L)
{
    return i < 0 ? i + L : (i >= L ? i - L : i);
}

__device__ __forceinline__ uint64_t live_mask(const Geom& g, int w)
{
    return (w == g.W - 1) ? (kSpinBits & ((g.rlast == kFields) ? ~0ull : ((1ull << (3 * g.rlast)) - 1ull)))
                          : kSpinBits;
}

// Block-wide sum of two counters, added with one atomic each to target[0..1].
__device__ __forceinline__ void block_add_counts(unsigned long long* target, uint32_t anti, uint32_t up)
{
    __shared__ unsigned int s_anti[32], s_up[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5;
    anti = __reduce_add_sync(0xffffffffu, anti);
    up = __reduce_add_sync(0xffffffffu, up);
    if (lane == 0) { s_anti[warp] = anti; s_up[warp] = up; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
        unsigned int a = (lane < nw) ? s_anti[lane] : 0u;
        unsigned int u = (lane < nw) ? s_up[lane] : 0u;
        a = __reduce_add_sync(0xffffffffu, a);
        u = __reduce_add_sync(0xffffffffu, u);
        if (lane == 0) {
            atomicAdd(target + 0, (unsigned long long)a);
            atomicAdd(target + 1, (unsigned long long)u);
        }
    }
}

// Accept bits of one field for one row.  A1 collects r < thr1 at bit K2 (the
// spin bit of the field within its 32-bit half), A0 collects r < thr0 at bit
// K2 + 1.  The inserts are predicated PTX, so a compare result never becomes
// a 0/1 value and the bit is an immediate: the r < thr1 insert is an OR on the
// ALU, the r < thr0 insert a multiply-add (K * one + A0) on the FMA pipe, which
// balances the two pipes against the Philox XORs (ALU) and multiplies (FMA).
template <int K2>
__device__ __forceinline__ void accept_insert(uint32_t& A1, uint32_t& A0, uint32_t r, uint32_t thr0,
                                              uint32_t thr1, uint32_t one)
{
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(A1) : "r"(r), "r"(thr1), "n"(1u << K2));
#if ISING_INSERTS_ON_ALU
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(A0) : "r"(r), "r"(thr0), "n"(2u << K2));
#else
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %4, %3, %0;\n\t}"
        : "+r"(A0) : "r"(r), "r"(thr0), "n"(2u << K2), "r"(one));
#endif
}

// Accumulators of one row: [0] r < thr1 bits of fields 0..10, [1] r < thr0
// (shifted up one bit) of fields 0..10, [2], [3] the same for fields 11..20.
struct AcceptBits {
    uint32_t a[4][4];   // [row][word]
};

// Fields k .. 20 of one Philox row group (compile-time k: immediate bit masks).
template <int k, int ROUNDS>
struct FieldLoop {
    __device__ __forceinline__ static void run(const PhiloxRowKey& pk, const PhiloxKeys& rk, uint32_t m0,
                                               AcceptBits& acc, uint32_t thr0, uint32_t thr1, uint32_t one)
    {
        uint32_t rnd[4];
        philox_row<ROUNDS>(pk, rk, m0 + (uint32_t)k, rnd);
        constexpr int half = k <= 10 ? 0 : 2;
        constexpr int K2 = k <= 10 ? 3 * k : 3 * k - 32;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            accept_insert<K2>(acc.a[e][half], acc.a[e][half + 1], rnd[e], thr0, thr1, one);
        FieldLoop<k + 1, ROUNDS>::run(pk, rk, m0, acc, thr0, thr1, one);
    }
};
template <int ROUNDS>
struct FieldLoop<kFields, ROUNDS> {
    __device__ __forceinline__ static void run(const PhiloxRowKey&, const PhiloxKeys&, uint32_t, AcceptBits&,
                                               uint32_t, uint32_t, uint32_t)
    {
    }
};

// The work of one thread: rows row0 .. row0+3 (those below L) of word column
// w of colour C, at sweep t (Sec. 2 steps 1-3 for every site of the colour at
// once; same-colour sites are never neighbours).  One Philox call covers the
// four rows of one field.
//
// Per row, with s the own word and u, d, h0, h1 the four aligned neighbour
// words, x_n = s ^ n has the spin bit of field k set iff neighbour n is
// anti-aligned (Eq. 3 summed bitwise instead of with carries):
//   any = x1|x2|x3|x4                     (a >= 1)
//   ge2 = x1&x2 | x3&x4 | (x1^x2)&(x3^x4) (a >= 2: dE <= 0, Table 1)
//   accept = ge2 | any & (r < thr1) | ~any & (r < thr0)
// GLOBAL selects read-only-cache loads (lattice in global memory) or plain
// loads (lattice in shared memory).  Offsets are 32-bit (L * pitch < 2^32).
// UPDATE = false skips the flip (measurement only).  RECORD adds the
// anti-aligned bond count of the (updated) colour-1 words and the up-spin
// count of both colours to anti / up: E = 2 anti - 2 L^2, M = 2 up - L^2.
template <int C, bool UPDATE, bool RECORD, bool GLOBAL = true, int ROUNDS = 10>
__device__ __forceinline__ void sweep_rows(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                           const Geom& g, int row0, int w, uint64_t t, const PhiloxKeys& rk,
                                           uint32_t thr0, uint32_t thr1, uint32_t all0w, uint32_t all1w,
                                           uint32_t one, uint32_t& anti, uint32_t& up)
{
    constexpr int ROWS = 4;
    const int nrows = min(ROWS, g.L - row0);
    const uint64_t live = live_mask(g, w);
    const uint32_t P = (uint32_t)g.P;
    const uint32_t base = (uint32_t)row0 * P + (uint32_t)w;
    const uint32_t up_off = row0 == 0 ? (uint32_t)(g.L - 1) * P + (uint32_t)w : base - P;
    const uint32_t dn_off = row0 + nrows >= g.L ? (uint32_t)w : base + (uint32_t)nrows * P;
    const uint32_t wl = (uint32_t)((w > 0) ? w - 1 : g.W - 1);
    const uint32_t wr = (uint32_t)((w < g.W - 1) ? w + 1 : 0);

    const uint64_t n = lattice_words(g);
    // All loads first: their latency overlaps the Philox work below.
    // oc[r] = other-colour row row0 - 1 + r (periodic), column w.
    uint64_t oc[ROWS + 2], sw[ROWS], side[ROWS];
    oc[0] = word_ld<GLOBAL>(other, up_off, n, __LINE__);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (r < nrows) {
            const uint32_t o = base + (uint32_t)r * P;
            oc[r + 1] = word_ld<GLOBAL>(other, o, n, __LINE__);
            sw[r] = word_ld<false>(own, o, n, __LINE__);
            const uint32_t os = o - (uint32_t)w + ((((r + C) & 1) == 0) ? wl : wr);   // row0 is a multiple of 4
            side[r] = word_ld<GLOBAL>(other, os, n, __LINE__);
        } else {
            oc[r + 1] = 0;
            sw[r] = 0;
            side[r] = 0;
        }
    }
    {
        const uint64_t dn = word_ld<GLOBAL>(other, dn_off, n, __LINE__);   // row below the last present row
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
            if (r + 1 == nrows) oc[r + 2] = dn;
        if (nrows == ROWS) oc[ROWS + 1] = dn;
    }

    AcceptBits acc;
#pragma unroll
    for (int e = 0; e < ROWS; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.a[e][q] = 0;
    if (UPDATE) {
        const uint32_t tl = (uint32_t)t;
        const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)C;
        const PhiloxRowKey pk = philox_row_key((uint32_t)(row0 >> 2), tl, th, rk);
        FieldLoop<0, ROUNDS>::run(pk, rk, (uint32_t)w * kFields, acc, thr0, thr1, one);
    }
    const uint64_t all0 = ((uint64_t)all0w << 32 | all0w) & live;
    const uint64_t all1 = ((uint64_t)all1w << 32 | all1w) & live;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (r < nrows) {
            const uint64_t s = sw[r];
            const uint64_t u = oc[r], d = oc[r + 2], h0 = oc[r + 1];
            // the other-colour word shifted by one field (horizontal neighbour at m -/+ 1)
            uint64_t h1;
            if (((r + C) & 1) == 0) {
                const int sh = (w > 0) ? 60 : 3 * (g.rlast - 1);
                h1 = (h0 << 3) | (side[r] >> sh);
            } else {
                const int sh = (w < g.W - 1) ? 60 : 3 * (g.rlast - 1);
                h1 = (h0 >> 3) | (side[r] << sh);
            }
            const uint64_t x1 = s ^ u, x2 = s ^ d, x3 = s ^ h0, x4 = s ^ h1;
            uint64_t s_new = s;
            if (UPDATE) {
                const uint64_t any = x1 | x2 | x3 | x4;
                const uint64_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
                const uint64_t c1 = ((uint64_t)acc.a[r][2] << 32 | acc.a[r][0]) | all1;
                const uint64_t c0 = (((uint64_t)acc.a[r][3] << 32 | acc.a[r][1]) >> 1) | all0;
                const uint64_t accept = ge2 | (any & c1) | (~any & c0);
                s_new = s ^ (accept & live);
                word_st(own, base + (uint32_t)r * P, s_new, n, __LINE__);
            }
            if (RECORD) {
                anti += __popcll((s_new ^ u) & live) + __popcll((s_new ^ d) & live)
                      + __popcll((s_new ^ h0) & live) + __popcll((s_new ^ h1) & live);
                up += __popcll(s_new & live) + __popcll(h0 & live);
            }
        }
    }
}

// ---- Split forms of sweep_rows -------------------------------------------
// The work of an item in two parts: its accept masks (the Philox draws
// against the thresholds; they depend on the site, sweep and colour only,
// never on the spins) and their application to the item's rows.  So the
// masks can be drawn by other threads than the ones that apply them, or
// before the spins they apply to exist: F lanes per item on the launch path
// for lattices too small to fill the GPU with one thread per item, and all
// masks of a run drawn beforehand for the on-chip path.  The draws and the
// accept rule are those of sweep_rows, so the results are bit-identical.  All
// lanes of a warp must call the lane forms (shuffles); an item past the end
// (`valid` = false) is drawn as item 0 and never applied.

// F lanes per item (F = 2, 4 or 8; aligned groups of the warp): lane q draws
// the fields k = q + jF, collects its accept bits at bit 3jF (compile-time
// positions), shifts them by 3q to bit 3k and OR-merges the F lanes' masks
// with shuffles.  Every lane of the group gets all masks.
template <int F, int ROUNDS = 10>
__device__ __forceinline__ void item_masks_lanes(const Geom& g, int item, int q, uint64_t t, int colour,
                                                 const PhiloxKeys& rk, uint32_t thr0, uint32_t thr1,
                                                 uint64_t a1[4], uint64_t a0[4])
{
    static_assert(F == 2 || F == 4 || F == 8, "F: 2, 4 or 8 lanes per item");
    constexpr int J = (kFields + F - 1) / F;
    const int grp = item / g.W;
    const int w = item - grp * g.W;
    const uint32_t tl = (uint32_t)t;
    const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)colour;
    const PhiloxRowKey pk = philox_row_key((uint32_t)grp, tl, th, rk);
#pragma unroll
    for (int e = 0; e < 4; ++e) a1[e] = a0[e] = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int k = q + j * F;
        if (k < kFields) {
            uint32_t r[4];
            philox_row<ROUNDS>(pk, rk, (uint32_t)(w * kFields + k), r);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (r[e] < thr1) a1[e] |= 1ull << (3 * j * F);
                if (r[e] < thr0) a0[e] |= 1ull << (3 * j * F);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        a1[e] <<= 3 * q;
        a0[e] <<= 3 * q;
    }
#pragma unroll
    for (int d = 1; d < F; d <<= 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            a1[e] |= __shfl_xor_sync(0xffffffffu, a1[e], d);
            a0[e] |= __shfl_xor_sync(0xffffffffu, a0[e], d);
        }
    }
}

// Apply the masks m1 (r < thr1) and m0 (r < thr0) of row i, word w of colour
// C: the spin logic of sweep_rows for one row.  all0 / all1 are the "always"
// masks (thresholds of 2^32) and live the row's live spin bits.  RECORD adds
// the row's anti-aligned bonds and up spins to anti / up (colour 1).
template <int C, bool RECORD>
__device__ __forceinline__ void row_apply(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                          const Geom& g, int i, int w, uint64_t live, uint64_t m1, uint64_t m0,
                                          uint64_t all0, uint64_t all1, uint32_t& anti, uint32_t& up)
{
    const uint32_t P = (uint32_t)g.P;
    const uint32_t o = (uint32_t)i * P;
    const uint64_t n = lattice_words(g);
    const uint64_t s = word_ld<false>(own, o + (uint32_t)w, n, __LINE__);
    const uint64_t u = word_ld<false>(other, (uint32_t)wrap_row(i - 1, g.L) * P + (uint32_t)w, n, __LINE__);
    const uint64_t d = word_ld<false>(other, (uint32_t)wrap_row(i + 1, g.L) * P + (uint32_t)w, n, __LINE__);
    const uint64_t h0 = word_ld<false>(other, o + (uint32_t)w, n, __LINE__);
    // horizontal neighbour at m - 1 ((i + C) even) or m + 1 (odd), as in sweep_rows
    const bool left = ((i + C) & 1) == 0;
    const int ws = left ? ((w > 0) ? w - 1 : g.W - 1) : ((w < g.W - 1) ? w + 1 : 0);
    const int sh = (left ? (w > 0) : (w < g.W - 1)) ? 60 : 3 * (g.rlast - 1);
    const uint64_t side = word_ld<false>(other, o + (uint32_t)ws, n, __LINE__);
    const uint64_t h1 = left ? ((h0 << 3) | (side >> sh)) : ((h0 >> 3) | (side << sh));
    const uint64_t x1 = s ^ u, x2 = s ^ d, x3 = s ^ h0, x4 = s ^ h1;
    const uint64_t any = x1 | x2 | x3 | x4;
    const uint64_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
    const uint64_t accept = ge2 | (any & (m1 | all1)) | (~any & (m0 | all0));
    const uint64_t s_new = s ^ (accept & live);
    word_st(own, o + (uint32_t)w, s_new, n, __LINE__);
    if (RECORD) {
        anti += __popcll((s_new ^ u) & live) + __popcll((s_new ^ d) & live)
              + __popcll((s_new ^ h0) & live) + __popcll((s_new ^ h1) & live);
        up += __popcll(s_new & live) + __popcll(h0 & live);
    }
}

// row_apply for one 32-bit half of the row: hf = 0 holds fields 0..10 (bits
// 0..31), hf = 1 fields 11..20 (bits 32..63); m1, m0, live, all0 and all1
// are that half of the row's words.  The two halves of a word are updated by
// different threads with 32-bit stores; the neighbour words of the other
// colour are read whole, since the shifted one carries a field across the
// halves.
template <int C, bool RECORD>
__device__ __forceinline__ void row_half_apply(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                               const Geom& g, int i, int w, int hf, uint32_t live, uint32_t m1,
                                               uint32_t m0, uint32_t all0, uint32_t all1, uint32_t& anti,
                                               uint32_t& up)
{
    const uint32_t P = (uint32_t)g.P;
    const uint32_t o = (uint32_t)i * P;
    const uint64_t n = lattice_words(g);
    uint32_t* own32 = reinterpret_cast<uint32_t*>(own);
    const uint32_t* other32 = reinterpret_cast<const uint32_t*>(other);
    const uint32_t s = half_ld(own32, 2 * (o + (uint32_t)w) + hf, 2 * n, __LINE__);
    const uint32_t u = half_ld(other32, 2 * ((uint32_t)wrap_row(i - 1, g.L) * P + (uint32_t)w) + hf, 2 * n, __LINE__);
    const uint32_t d = half_ld(other32, 2 * ((uint32_t)wrap_row(i + 1, g.L) * P + (uint32_t)w) + hf, 2 * n, __LINE__);
    const uint64_t h0w = word_ld<false>(other, o + (uint32_t)w, n, __LINE__);
    // horizontal neighbour at m - 1 ((i + C) even) or m + 1 (odd), as in sweep_rows
    const bool left = ((i + C) & 1) == 0;
    const int ws = left ? ((w > 0) ? w - 1 : g.W - 1) : ((w < g.W - 1) ? w + 1 : 0);
    const int sh = (left ? (w > 0) : (w < g.W - 1)) ? 60 : 3 * (g.rlast - 1);
    const uint64_t side = word_ld<false>(other, o + (uint32_t)ws, n, __LINE__);
    const uint64_t h1w = left ? ((h0w << 3) | (side >> sh)) : ((h0w >> 3) | (side << sh));
    const uint32_t h0 = (uint32_t)(h0w >> (32 * hf)), h1 = (uint32_t)(h1w >> (32 * hf));
    const uint32_t x1 = s ^ u, x2 = s ^ d, x3 = s ^ h0, x4 = s ^ h1;
    const uint32_t any = x1 | x2 | x3 | x4;
    const uint32_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
    const uint32_t accept = ge2 | (any & (m1 | all1)) | (~any & (m0 | all0));
    const uint32_t s_new = s ^ (accept & live);
    half_st(own32, 2 * (o + (uint32_t)w) + hf, s_new, 2 * n, __LINE__);
    if (RECORD) {
        anti += __popc((s_new ^ u) & live) + __popc((s_new ^ d) & live) + __popc((s_new ^ h0) & live)
              + __popc((s_new ^ h1) & live);
        up += __popc(s_new & live) + __popc(h0 & live);
    }
}

// Apply the masks of an item of colour C: lane q of its group of F lanes
// updates rows q, q + F, ... below 4 (one code path for all lanes, the row's
// masks picked by selection).  RECORD adds the item's
// anti-aligned bonds and up spins to anti / up (colour 1).
template <int C, bool RECORD, int F>
__device__ __forceinline__ void item_apply(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                           const Geom& g, int item, bool valid, int q, const uint64_t a1[4],
                                           const uint64_t a0[4], uint32_t all0w, uint32_t all1w, uint32_t& anti,
                                           uint32_t& up)
{
    constexpr int STEP = F < 4 ? F : 4;
    if (!valid) return;
    const int grp = item / g.W;
    const int w = item - grp * g.W;
    const int row0 = grp * 4;
    const uint64_t live = live_mask(g, w);
    const uint64_t all0 = ((uint64_t)all0w << 32 | all0w) & live;
    const uint64_t all1 = ((uint64_t)all1w << 32 | all1w) & live;
#pragma unroll
    for (int e0 = 0; e0 < 4; e0 += STEP) {
        const int e = e0 + q;
        if (e >= 4 || e >= g.L - row0) break;
        const uint64_t m1 = e == 0 ? a1[0] : (e == 1 ? a1[1] : (e == 2 ? a1[2] : a1[3]));
        const uint64_t m0 = e == 0 ? a0[0] : (e == 1 ? a0[1] : (e == 2 ? a0[2] : a0[3]));
        row_apply<C, RECORD>(own, other, g, row0 + e, w, live, m1, m0, all0, all1, anti, up);
    }
}

// All accept masks of one item drawn by one thread, with the draws and
// accumulators of sweep_rows, packed one word per row: packed[e] has r < thr1
// of field k at bit 3k and r < thr0 at bit 3k + 1.  For row_apply, m1 =
// packed and m0 = packed >> 1: their other bits fall on no spin bit.
template <int ROUNDS = 10>
__device__ __forceinline__ void item_masks_thread(const Geom& g, int item, uint64_t t, int colour,
                                                  const PhiloxKeys& rk, uint32_t thr0, uint32_t thr1, uint32_t one,
                                                  uint64_t packed[4])
{
    const int grp = item / g.W;
    const int w = item - grp * g.W;
    AcceptBits acc;
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.a[e][q] = 0;
    const uint32_t tl = (uint32_t)t;
    const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)colour;
    const PhiloxRowKey pk = philox_row_key((uint32_t)grp, tl, th, rk);
    FieldLoop<0, ROUNDS>::run(pk, rk, (uint32_t)w * kFields, acc, thr0, thr1, one);
#pragma unroll
    for (int e = 0; e < 4; ++e)
        packed[e] = (uint64_t)(acc.a[e][2] | acc.a[e][3]) << 32 | (acc.a[e][0] | acc.a[e][1]);
}

// Masks of an item with F lanes; an item past the end is drawn as item 0.
template <int F, int ROUNDS = 10>
__device__ __forceinline__ void item_masks(const Geom& g, int item, bool valid, int q, uint64_t t, int colour,
                                           const PhiloxKeys& rk, uint32_t thr0, uint32_t thr1, uint64_t a1[4],
                                           uint64_t a0[4])
{
    if (!valid) item = 0;
    item_masks_lanes<F, ROUNDS>(g, item, q, t, colour, rk, thr0, thr1, a1, a0);
}

// Draw and apply in one step (the launch path's lanes kernel).
template <int C, bool RECORD, int F, int ROUNDS = 10>
__device__ __forceinline__ void sweep_item_lanes(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                                 const Geom& g, int item, bool valid, int q, uint64_t t,
                                                 const PhiloxKeys& rk, uint32_t thr0, uint32_t thr1,
                                                 uint32_t all0w, uint32_t all1w, uint32_t& anti, uint32_t& up)
{
    uint64_t a1[4], a0[4];
    item_masks<F, ROUNDS>(g, item, valid, q, t, C, rk, thr0, thr1, a1, a0);
    item_apply<C, RECORD, F>(own, other, g, item, valid, q, a1, a0, all0w, all1w, anti, up);
}

// One half-sweep of colour C over one lattice.  LINEAR: a 1-D grid whose
// thread k owns item k = group * W + w (word w of rows 4 group .. 4 group + 3),
// so no thread idles on padding columns and the blocks tile the lattice
// without a partial column of blocks.  Otherwise thread (x, y) of a 2-D grid
// owns word column x and rows 4y .. 4y+3.  At most 256 threads per block.
// ROUNDS: Philox rounds of the draws (10, or the opt-in 7).
template <int C, bool UPDATE, bool RECORD, int ROUNDS = 10, bool LINEAR = true>
__global__ void __launch_bounds__(256, 3)
half_sweep_kernel(uint64_t* __restrict__ own, const uint64_t* __restrict__ other, Geom g, SweepArgs a)
{
    pdl_enter();
    int w, row0;
    if (LINEAR) {
        const uint32_t item = blockIdx.x * blockDim.x + threadIdx.x;
        const uint32_t grp = item / (uint32_t)g.W;
        w = (int)(item - grp * (uint32_t)g.W);
        row0 = (int)grp * 4;
    } else {
        w = blockIdx.x * blockDim.x + threadIdx.x;
        row0 = (blockIdx.y * blockDim.y + threadIdx.y) * 4;
    }
    uint32_t anti = 0, up = 0;
    if (w < g.W && row0 < g.L) {
        const uint64_t t = UPDATE ? *a.t_base + a.t_off : 0;
        sweep_rows<C, UPDATE, RECORD, true, ROUNDS>(own, other, g, row0, w, t, a.rk, a.thr0, a.thr1, a.all0,
                                                    a.all1, a.one, anti, up);
    }
    if (RECORD) {
        const int slot = (blockIdx.x + gridDim.x * blockIdx.y) % kCountSlots;
        block_add_counts(record_counts(a) + 2 * slot, anti, up);
    }
}

}  // namespace ising

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
#include <cstdint>
#include "philox.cuh"

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
    uint32_t key0, key1;       // Philox key = (lo32(seed), hi32(seed))
    uint32_t thr0, thr1;       // integer thresholds clamped to 2^32 - 1 ...
    uint32_t all0, all1;       // ... and ~0u where the threshold is 2^32
    unsigned long long* counts;  // E/M count slots of this record (RECORD only)
};

__device__ __forceinline__ int wrap_row(int i, int L)
{
    return i < 0 ? i + L : (i >= L ? i - L : i);
}

__device__ __forceinline__ uint64_t live_mask(const Geom& g, int w)
{
    return (w == g.W - 1) ? (kSpinBits & ((g.rlast == kFields) ? ~0ull : ((1ull << (3 * g.rlast)) - 1ull)))
                          : kSpinBits;
}

// Other-colour word aligned so that field k holds the horizontal neighbour
// at m - 1 (dir = 0) or m + 1 (dir = 1) of field k of word w.
__device__ __forceinline__ uint64_t side_word(const uint64_t* __restrict__ orow, const Geom& g,
                                             int w, uint64_t center, int dir)
{
    if (dir == 0) {
        const int wp = (w > 0) ? w - 1 : g.W - 1;
        const int sh = (w > 0) ? 60 : 3 * (g.rlast - 1);
        return (center << 3) | (__ldg(orow + wp) >> sh);
    } else {
        const int wn = (w < g.W - 1) ? w + 1 : 0;
        const int sh = (w < g.W - 1) ? 60 : 3 * (g.rlast - 1);
        return (center >> 3) | (__ldg(orow + wn) << sh);
    }
}

// Block-wide sum of two counters into slot (blockIdx % kCountSlots) of `counts`.
__device__ __forceinline__ void block_add_counts(unsigned long long* counts, uint32_t anti, uint32_t up)
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
            const int slot = (blockIdx.x + gridDim.x * blockIdx.y) % kCountSlots;
            atomicAdd(counts + 2 * slot + 0, (unsigned long long)a);
            atomicAdd(counts + 2 * slot + 1, (unsigned long long)u);
        }
    }
}

// One Metropolis half-sweep of colour C (Sec. 2 steps 1-3 for every site of
// the colour at once; same-colour sites are never neighbours).  A thread owns
// ROWS consecutive rows (a multiple of 4: one Philox call covers the four
// rows 4g..4g+3 of one field) of one word column.
//
// Per row, with s the own word and u, d, h0, h1 the four aligned neighbour
// words, x_n = s ^ n has the spin bit of field k set iff neighbour n is
// anti-aligned (Eq. 3 summed bitwise instead of with carries):
//   any = x1|x2|x3|x4                     (a >= 1)
//   ge2 = x1&x2 | x3&x4 | (x1^x2)&(x3^x4) (a >= 2: dE <= 0, Table 1)
//   accept = ge2 | any & (r < thr1) | ~any & (r < thr0)
// UPDATE = false skips the flip (measurement only).  RECORD adds the
// anti-aligned bond count of the (updated) colour-1 words and the up-spin
// count of both colours to the count slots: E = 2 anti - 2 L^2, M = 2 up - L^2.
template <int ROWS, int C, bool UPDATE, bool RECORD>
__global__ void __launch_bounds__(512)
half_sweep_kernel(uint64_t* __restrict__ own, const uint64_t* __restrict__ other, Geom g, SweepArgs a)
{
    static_assert(ROWS % 4 == 0, "ROWS must be a multiple of 4");
    constexpr int NG = ROWS / 4;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int row0 = (blockIdx.y * blockDim.y + threadIdx.y) * ROWS;
    const bool active = (w < g.W) && (row0 < g.L);
    uint32_t anti = 0, up = 0;

    if (active) {
        const int nrows = min(ROWS, g.L - row0);
        const uint64_t live = live_mask(g, w);

        uint64_t acc0[ROWS], acc1[ROWS];
        if (UPDATE) {
            const uint64_t t = *a.t_base + a.t_off;
            const uint32_t tl = (uint32_t)t;
            const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)C;
            PhiloxRowKey pk[NG];
#pragma unroll
            for (int q = 0; q < NG; ++q)
                pk[q] = philox_row_key((uint32_t)(row0 / 4 + q), tl, th, a.key0, a.key1);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) { acc0[r] = 0; acc1[r] = 0; }
            const uint32_t m0 = (uint32_t)w * kFields;
#pragma unroll
            for (int k = 0; k < kFields; ++k) {
#pragma unroll
                for (int q = 0; q < NG; ++q) {
                    uint32_t rnd[4];
                    philox_row(pk[q], m0 + (uint32_t)k, rnd);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        acc0[4 * q + e] |= (uint64_t)(rnd[e] < a.thr0) << (3 * k);
                        acc1[4 * q + e] |= (uint64_t)(rnd[e] < a.thr1) << (3 * k);
                    }
                }
            }
        }

        // Other-colour rows row0-1 .. row0+nrows (center column w).
        uint64_t oc[ROWS + 2];
#pragma unroll
        for (int r = 0; r < ROWS + 2; ++r) {
            if (r <= nrows + 1) {
                const int i = wrap_row(row0 - 1 + r, g.L);
                oc[r] = __ldg(other + (size_t)i * g.P + w);
            } else {
                oc[r] = 0;
            }
        }
        const uint64_t all0 = ((uint64_t)a.all0 << 32 | a.all0) & live;
        const uint64_t all1 = ((uint64_t)a.all1 << 32 | a.all1) & live;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (r < nrows) {
                const int i = row0 + r;
                uint64_t* srow = own + (size_t)i * g.P;
                const uint64_t s = srow[w];
                const uint64_t u = oc[r], d = oc[r + 2], h0 = oc[r + 1];
                const int dir = (r + C) & 1;   // row0 is a multiple of 4
                const uint64_t h1 = side_word(other + (size_t)i * g.P, g, w, h0, dir);
                const uint64_t x1 = s ^ u, x2 = s ^ d, x3 = s ^ h0, x4 = s ^ h1;
                uint64_t s_new = s;
                if (UPDATE) {
                    const uint64_t any = x1 | x2 | x3 | x4;
                    const uint64_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
                    const uint64_t c0 = acc0[r] | all0;
                    const uint64_t c1 = acc1[r] | all1;
                    const uint64_t accept = ge2 | (any & c1) | (~any & c0);
                    s_new = s ^ (accept & live);
                    srow[w] = s_new;
                }
                if (RECORD) {
                    anti += __popcll((s_new ^ u) & live) + __popcll((s_new ^ d) & live)
                          + __popcll((s_new ^ h0) & live) + __popcll((s_new ^ h1) & live);
                    up += __popcll(s_new & live) + __popcll(h0 & live);
                }
            }
        }
    }
    if (RECORD)
        block_add_counts(a.counts, anti, up);
}

}  // namespace ising

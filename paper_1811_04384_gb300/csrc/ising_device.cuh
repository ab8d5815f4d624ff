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
    uint32_t thr0, thr1;       // integer thresholds clamped to 2^32 - 1 ...
    uint32_t all0, all1;       // ... and ~0u where the threshold is 2^32
    uint32_t one;              // the value 1, as a launch operand (see accept_insert)
    PhiloxKeys rk;             // round keys of the key (lo32(seed), hi32(seed))
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

// Set the bit of field k in the accept masks A0 (r < thr0) and A1 (r < thr1).
// The two inserts are written as predicated PTX so that the compare result
// never becomes a 0/1 value: the first is a multiply-add (K * one + A0, which
// runs on the FMA pipe), the second an OR on the ALU, balancing the two pipes
// against the Philox multiplies (FMA) and XORs (ALU).
__device__ __forceinline__ void accept_insert(uint32_t& A0, uint32_t& A1, uint32_t r, uint32_t thr0,
                                              uint32_t thr1, uint32_t K, uint32_t one)
{
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
        : "+r"(A0) : "r"(r), "r"(thr0), "r"(K), "r"(one));
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(A1) : "r"(r), "r"(thr1), "r"(K));
}

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
// loads (lattice in shared memory).
// UPDATE = false skips the flip (measurement only).  RECORD adds the
// anti-aligned bond count of the (updated) colour-1 words and the up-spin
// count of both colours to anti / up: E = 2 anti - 2 L^2, M = 2 up - L^2.
template <int C, bool UPDATE, bool RECORD, bool GLOBAL = true>
__device__ __forceinline__ void sweep_rows(uint64_t* __restrict__ own, const uint64_t* __restrict__ other,
                                           const Geom& g, int row0, int w, uint64_t t, const PhiloxKeys& rk,
                                           uint32_t thr0, uint32_t thr1, uint32_t all0w, uint32_t all1w,
                                           uint32_t one, uint32_t& anti, uint32_t& up)
{
    constexpr int ROWS = 4;
    const int nrows = min(ROWS, g.L - row0);
    const uint64_t live = live_mask(g, w);

    // All loads first: their latency overlaps the Philox work below.
    uint64_t oc[ROWS + 2], sw[ROWS], side[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS + 2; ++r) {
        if (r <= nrows + 1) {
            const int i = wrap_row(row0 - 1 + r, g.L);
            oc[r] = GLOBAL ? __ldg(other + (size_t)i * g.P + w) : other[(size_t)i * g.P + w];
        } else {
            oc[r] = 0;
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (r < nrows) {
            const int i = row0 + r;
            sw[r] = own[(size_t)i * g.P + w];
            const int dir = (r + C) & 1;     // row0 is a multiple of 4
            const int wn = dir == 0 ? ((w > 0) ? w - 1 : g.W - 1) : ((w < g.W - 1) ? w + 1 : 0);
            side[r] = GLOBAL ? __ldg(other + (size_t)i * g.P + wn) : other[(size_t)i * g.P + wn];
        } else {
            sw[r] = 0;
            side[r] = 0;
        }
    }

    uint32_t lo0[ROWS] = {0, 0, 0, 0}, hi0[ROWS] = {0, 0, 0, 0};
    uint32_t lo1[ROWS] = {0, 0, 0, 0}, hi1[ROWS] = {0, 0, 0, 0};
    if (UPDATE) {
        const uint32_t tl = (uint32_t)t;
        const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)C;
        const PhiloxRowKey pk = philox_row_key((uint32_t)(row0 >> 2), tl, th, rk);
        const uint32_t m0 = (uint32_t)w * kFields;
#pragma unroll
        for (int k = 0; k < kFields; ++k) {
            uint32_t rnd[4];
            philox_row(pk, rk, m0 + (uint32_t)k, rnd);
            // field k: bit 3k of the word; fields 0..10 in the low half, 11..20 in the high half
            const uint32_t K = (k <= 10) ? (1u << (3 * k)) : (1u << (3 * k - 32));
#pragma unroll
            for (int e = 0; e < ROWS; ++e) {
                if (k <= 10) accept_insert(lo0[e], lo1[e], rnd[e], thr0, thr1, K, one);
                else accept_insert(hi0[e], hi1[e], rnd[e], thr0, thr1, K, one);
            }
        }
    }
    const uint64_t all0 = ((uint64_t)all0w << 32 | all0w) & live;
    const uint64_t all1 = ((uint64_t)all1w << 32 | all1w) & live;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (r < nrows) {
            const int i = row0 + r;
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
                const uint64_t c0 = ((uint64_t)hi0[r] << 32 | lo0[r]) | all0;
                const uint64_t c1 = ((uint64_t)hi1[r] << 32 | lo1[r]) | all1;
                const uint64_t accept = ge2 | (any & c1) | (~any & c0);
                s_new = s ^ (accept & live);
                own[(size_t)i * g.P + w] = s_new;
            }
            if (RECORD) {
                anti += __popcll((s_new ^ u) & live) + __popcll((s_new ^ d) & live)
                      + __popcll((s_new ^ h0) & live) + __popcll((s_new ^ h1) & live);
                up += __popcll(s_new & live) + __popcll(h0 & live);
            }
        }
    }
}

// One half-sweep of colour C over one lattice: thread (x, y) of the grid owns
// word column x and rows 4y .. 4y+3.  At most 256 threads per block.
template <int C, bool UPDATE, bool RECORD>
__global__ void __launch_bounds__(256, 3)
half_sweep_kernel(uint64_t* __restrict__ own, const uint64_t* __restrict__ other, Geom g, SweepArgs a)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int row0 = (blockIdx.y * blockDim.y + threadIdx.y) * 4;
    uint32_t anti = 0, up = 0;
    if (w < g.W && row0 < g.L) {
        const uint64_t t = UPDATE ? *a.t_base + a.t_off : 0;
        sweep_rows<C, UPDATE, RECORD>(own, other, g, row0, w, t, a.rk, a.thr0, a.thr1, a.all0, a.all1,
                                      a.one, anti, up);
    }
    if (RECORD) {
        const int slot = (blockIdx.x + gridDim.x * blockIdx.y) % kCountSlots;
        block_add_counts(a.counts + 2 * slot, anti, up);
    }
}

}  // namespace ising

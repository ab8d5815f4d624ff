// The paper's own multi-spin layout (Sec. 3, Fig. 1-2): the L x L lattice,
// L = 21 N, becomes an N x L lattice of words; word S(I, J) holds the spins
// s(I + kN, J), k = 0..20, in field k (bits 3k..3k+2).  Every neighbour of
// field k sits in field k of the neighbouring word, except across the top
// and bottom word rows, where the neighbour word is rotated by one field
// (Sec. 3, Fig. 2).  With N even all 21 spins of a word share one colour,
// (I + J) & 1, so the checkerboard update works word by word.
//
// The sweep uses Eq. 3 in its arithmetic form: the 3-bit field sums of the
// four XORs give a = 0..4 without carries; a >= 2 always flips, a = 0 / 1
// flips iff the site's draw is below thr[a].  The draws are the sites' own
// Philox values (the same keying as the row-packed path), so the chain is
// identical: the layout changes where spins live, not what happens to them.
// Needs N % 4 == 0 (L % 84 == 0): then the four word rows 4q..4q+3 of one
// field k are the rows of one Philox row group, and one call serves them.
#include <cuda_runtime.h>

#include "ising_interleaved.h"
#include "ising_interleaved.cuh"
#include "ising_internal.h"

namespace ising {
namespace {

// Hot start: field k of S(I, J) is +1 iff the Philox draw at t = 0 of site
// (I + kN, J) is below 2^31.  One thread per word.
__global__ void ci_init_hot_kernel(uint64_t* __restrict__ S, int L, int N, uint32_t k0, uint32_t k1)
{
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    const int I = blockIdx.y * blockDim.y + threadIdx.y;
    if (J >= L || I >= N) return;
    uint64_t word = 0;
    for (int k = 0; k < 21; ++k) {
        const int i = I + k * N;
        uint32_t x[4] = {(uint32_t)(i >> 2), (uint32_t)(J >> 1), 0u, (uint32_t)((i + J) & 1)};
        philox10(x, k0, k1);
        word |= (uint64_t)((x[i & 3] >> 31) ^ 1u) << (3 * k);
    }
    S[(size_t)I * L + J] = word;
}

__global__ void ci_fill_kernel(uint64_t* __restrict__ S, size_t n, uint64_t v)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) S[k] = v;
}

__global__ void ci_pack_kernel(uint64_t* __restrict__ S, int L, int N, const int8_t* __restrict__ s)
{
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    const int I = blockIdx.y * blockDim.y + threadIdx.y;
    if (J >= L || I >= N) return;
    uint64_t word = 0;
    for (int k = 0; k < 21; ++k)
        word |= (uint64_t)(s[(size_t)(I + k * N) * L + J] > 0) << (3 * k);
    S[(size_t)I * L + J] = word;
}

__global__ void ci_unpack_kernel(const uint64_t* __restrict__ S, int L, int N, int8_t* __restrict__ s)
{
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    const int I = blockIdx.y * blockDim.y + threadIdx.y;
    if (J >= L || I >= N) return;
    const uint64_t word = S[(size_t)I * L + J];
    for (int k = 0; k < 21; ++k)
        s[(size_t)(I + k * N) * L + J] = ((word >> (3 * k)) & 1ull) ? (int8_t)1 : (int8_t)-1;
}

// The masks of ci_half_sweep_kernel for the sweeps j = 0 .. nsweeps-1 after
// sweep (t_base ? *t_base : 0) + t0, drawn ahead on all SMs: one thread per
// (j, colour, q, m), masks[(((j * 2 + colour) * N/4 + q) * L/2 + m) * 4 + e]
// = packed masks of word row 4q + e.
template <int ROUNDS>
__global__ void __launch_bounds__(128)
ci_mask_draw_kernel(int L, int N, SweepArgs a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                    uint64_t* __restrict__ masks)
{
    const long long Q = N / 4, M = L / 2;
    const long long total = (long long)nsweeps * 2 * Q * M;
    const uint64_t tb = (t_base ? *t_base : 0) + t0 + 1;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(k % M);
        const int q = (int)((k / M) % Q);
        const int colour = (int)((k / (M * Q)) & 1);
        const int j = (int)(k / (2 * M * Q));
        uint64_t packed[4];
        ci_masks<ROUNDS>(N, q, m, tb + (uint64_t)j, colour, a, packed);
#pragma unroll
        for (int e = 0; e < 4; ++e) masks[(size_t)k * 4 + e] = packed[e];
    }
}

// One half-sweep of colour C.  Thread (m, q) owns word rows 4q .. 4q+3 and the
// column pair 2m, 2m+1; in each row it updates the colour-C word
// J_e = 2m + ((I_e + C) & 1).  Its accept masks come from ci_masks, or with
// PRE from `masks` (this sweep and colour's block of ci_mask_draw_kernel).
// RECORD (colour 1) also counts the anti-aligned bonds of the four colour-1
// words and the up spins of all eight words of the block.
template <int C, bool UPDATE, bool RECORD, int ROUNDS, bool PRE = false>
__global__ void __launch_bounds__(128)
ci_half_sweep_kernel(uint64_t* __restrict__ S, int L, int N, SweepArgs a, const uint64_t* __restrict__ masks)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y * blockDim.y + threadIdx.y;
    uint32_t anti = 0, up = 0;
    if (m < L / 2 && q < N / 4) {
        const uint64_t n = (uint64_t)N * L;
        uint64_t s[4], xl[4], xr[4], xu[4], xd[4], other[4];
        int J[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int I = 4 * q + e;
            J[e] = 2 * m + ((I + C) & 1);
            const int Jl = J[e] == 0 ? L - 1 : J[e] - 1;
            const int Jr = J[e] == L - 1 ? 0 : J[e] + 1;
            const uint64_t row = (uint64_t)I * L;
            s[e] = word_ld<false>(S, row + J[e], n, __LINE__);
            xl[e] = word_ld<true>(S, row + Jl, n, __LINE__);
            xr[e] = word_ld<true>(S, row + Jr, n, __LINE__);
            other[e] = (J[e] & 1) ? xl[e] : xr[e];    // the other word of the column pair
            xu[e] = I == 0 ? rotate_up(word_ld<true>(S, (uint64_t)(N - 1) * L + J[e], n, __LINE__))
                           : word_ld<true>(S, (uint64_t)(I - 1) * L + J[e], n, __LINE__);
            xd[e] = I == N - 1 ? rotate_down(word_ld<true>(S, (uint64_t)J[e], n, __LINE__))
                               : word_ld<true>(S, (uint64_t)(I + 1) * L + J[e], n, __LINE__);
        }
        // c1: r < thr1 at the spin bits; c0 >> 1 of the same word: r < thr0 there
        // (its other bits fall on no spin bit and are masked below)
        uint64_t c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
        if (UPDATE) {
            uint64_t packed[4];
            if (PRE) {
#pragma unroll
                for (int e = 0; e < 4; ++e) packed[e] = __ldg(masks + ((size_t)q * (L / 2) + m) * 4 + e);
            } else {
                ci_masks<ROUNDS>(N, q, m, *a.t_base + a.t_off, C, a, packed);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                c1[e] = packed[e];
                c0[e] = packed[e] >> 1;
            }
        }
        const uint64_t all0 = ((uint64_t)a.all0 << 32 | a.all0) & kAllFields;
        const uint64_t all1 = ((uint64_t)a.all1 << 32 | a.all1) & kAllFields;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int I = 4 * q + e;
            uint64_t sn = s[e];
            if (UPDATE) {
                // Eq. 3: each XOR field is 0/1, so the 3-bit sums hold a = 0..4 without carries
                const uint64_t A = (s[e] ^ xu[e]) + (s[e] ^ xd[e]) + (s[e] ^ xl[e]) + (s[e] ^ xr[e]);
                const uint64_t ge2 = ((A >> 1) | (A >> 2)) & kAllFields;           // a >= 2: dE <= 0
                const uint64_t any = (A | (A >> 1) | (A >> 2)) & kAllFields;       // a >= 1
                const uint64_t accept = ge2 | (any & (c1[e] | all1)) | (~any & (c0[e] | all0));
                sn = s[e] ^ (accept & kAllFields);
                word_st(S, (uint64_t)I * L + J[e], sn, n, __LINE__);
            }
            if (RECORD) {
                anti += __popcll(sn ^ xu[e]) + __popcll(sn ^ xd[e]) + __popcll(sn ^ xl[e]) + __popcll(sn ^ xr[e]);
                up += __popcll(sn) + __popcll(other[e]);
            }
        }
    }
    if (RECORD) {
        const int slot = (blockIdx.x + gridDim.x * blockIdx.y) % kCountSlots;
        block_add_counts(record_counts(a) + 2 * slot, anti, up);
    }
}

// ---- The paper's own chain: random memory words (Sec. 4-5, Appendix A) ----
// One phase of one Monte Carlo iteration: each block is one strip (the
// paper's process) and runs that strip's sequence of 10 N h word updates on
// its half strip [col0, col0 + h) in sequence order, where update s picks
// the word drawn from (seed, t, phase, strip, s) and applies the Metropolis
// rule to its 21 spins.  Strips of one phase touch no common or neighbouring
// words, so the blocks are independent.
//
// Within a strip the updates run as a window of kRwWindow pending ones, in
// sequence order (slot 0 the oldest).  In each round every pending update
// whose word and four neighbour words no older pending update touches runs;
// the others wait for the next round, and the freed slots take the next
// updates of the sequence.  An update that runs has every older update on
// its word or a neighbouring word already applied, and none of the updates
// of one round reads a word another one writes, so the result is the
// sequential chain's, word for word.  The oldest pending update can always
// run, so every round makes progress and the loop ends after at most 10 N h
// rounds.  "Touches" is tracked in a shared-memory table of kRwBuckets
// claims indexed by the word's index in the half strip modulo kRwBuckets: two
// words sharing a bucket only make an update wait longer, never run early.
//
// An update's draws (the chosen word and the accept masks of its 21 spins)
// depend on its counter only.  ci_rw_draw_kernel makes those of a whole
// iteration beforehand on all SMs (PRE), so a window slot only loads them;
// lattices whose draws would pass kRwDrawBytesMax draw them in the block
// instead, when an update enters the window.  With WIN the block keeps its
// half strip and the two columns beside it in shared memory for the phase
// (the columns beside it are not updated in this phase), so a round touches
// no global memory; strips too wide for shared memory work on the lattice in
// global memory.
constexpr int kRwWindow = 256;
constexpr int kRwRing = 4 * kRwWindow;                  // pre-drawn updates staged ahead in shared memory
constexpr int kRwBuckets = 8192;
constexpr size_t kRwWinBytesMax = 160 * 1024;         // dynamic shared memory of the WIN form
constexpr size_t kRwDrawBytesMax = (size_t)256 << 20;  // pre-drawn updates of one iteration

// The 24 draw words of update `step` (6 Philox4x32-10 blocks) reduced to
// the chosen word (row I, column jr of the half strip) and the accept masks
// packed in one word: draw < thr1 at the spin bit of field k, draw < thr0
// one bit above it.
__device__ __forceinline__ void rw_draw(const SweepArgs& a, uint32_t step, uint32_t strip, uint32_t tl,
                                        uint32_t x3, int N, int h, uint32_t& I, uint32_t& jr, uint64_t& packed)
{
    uint32_t w[24];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        uint32_t x0 = step, x1 = strip * 8u + (uint32_t)b, x2 = tl, y3 = x3;
#pragma unroll
        for (int r = 0; r < 10; ++r) philox_round(x0, x1, x2, y3, a.rk.k0[r], a.rk.k1[r]);
        w[4 * b] = x0; w[4 * b + 1] = x1; w[4 * b + 2] = x2; w[4 * b + 3] = y3;
    }
    I = __umulhi(w[0], (uint32_t)N);
    jr = __umulhi(w[1], (uint32_t)h);
    uint64_t m = 0;
#pragma unroll
    for (int k = 0; k < 21; ++k)
        m |= (uint64_t)(w[2 + k] < a.thr1) << (3 * k) | (uint64_t)(w[2 + k] < a.thr0) << (3 * k + 1);
    packed = m;
}

// All updates of iteration *t_base + t_off, both phases: entry
// draws[phase base + q * U_p + s] = (I << 16 | column in the half strip,
// packed masks) for update s of strip q; phase 0's entries first.
__global__ void __launch_bounds__(128)
ci_rw_draw_kernel(int L, int N, int NC, int nstrips, SweepArgs a, ulonglong2* __restrict__ draws)
{
    const int h0 = NC / 2, h1 = NC - NC / 2;
    const uint64_t U0 = 10ull * N * h0, U1 = 10ull * N * h1;
    const uint64_t n0 = U0 * nstrips, total = n0 + U1 * nstrips;
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int phase = k < n0 ? 0 : 1;
    const uint64_t r = phase ? k - n0 : k;
    const uint64_t U = phase ? U1 : U0;
    const uint32_t q = (uint32_t)(r / U), step = (uint32_t)(r - (uint64_t)q * U);
    const uint64_t t = *a.t_base + a.t_off;
    const uint32_t x3 = 0x80000000u | ((uint32_t)(t >> 32) << 1) | (uint32_t)phase;
    uint32_t I, jr;
    uint64_t packed;
    rw_draw(a, step, q, (uint32_t)t, x3, N, phase ? h1 : h0, I, jr, packed);
    draws[k] = make_ulonglong2((uint64_t)(I << 16 | jr), packed);
}

// 16 bytes global -> shared, asynchronously.
__device__ __forceinline__ void ring_copy(ulonglong2* smem_dst, const ulonglong2* gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

template <bool PRE, bool WIN>
__global__ void __launch_bounds__(kRwWindow)
ci_rw_phase_kernel(uint64_t* S, int L, int N, int NC, int phase, SweepArgs a, const ulonglong2* __restrict__ draws)
{
    __shared__ uint32_t claim[kRwBuckets];
    __shared__ uint32_t sl_word[2][kRwWindow];          // I << 16 | column in the half strip
    __shared__ uint64_t sl_mask[2][kRwWindow];          // packed masks
    __shared__ uint32_t warp_keep[kRwWindow / 32];
    __shared__ __align__(16) ulonglong2 ring[PRE ? kRwRing : 1];   // PRE: draws of steps next .. next + kRwRing - 1
    extern __shared__ __align__(16) uint64_t win[];     // WIN: N rows x (h + 2) words
    const int tid = threadIdx.x;
    const uint32_t q = blockIdx.x;
    const int h = phase == 0 ? NC / 2 : NC - NC / 2;
    const int col0 = (int)q * NC + (phase == 0 ? 0 : NC / 2);
    const uint32_t U = 10u * (uint32_t)N * (uint32_t)h;
    const uint64_t t = *a.t_base + a.t_off;
    const uint32_t tl = (uint32_t)t;
    const uint32_t x3 = 0x80000000u | ((uint32_t)(t >> 32) << 1) | (uint32_t)phase;
    const ulonglong2* my_draws = PRE ? draws + (size_t)q * U : nullptr;   // this phase's block of draws
    const uint64_t all1 = ((uint64_t)a.all1 << 32 | a.all1) & kAllFields;
    const uint64_t all0 = ((uint64_t)a.all0 << 32 | a.all0) & kAllFields;
    constexpr uint32_t B = kRwBuckets - 1;
    const int hw = h + 2;                                // window row: the column before, h, the column after
    const uint64_t n_lat = (uint64_t)N * L, n_win = (uint64_t)N * hw;
    for (int i = tid; i < kRwBuckets; i += kRwWindow) claim[i] = 0xFFFFFFFFu;
    if (WIN) {
        for (int idx = tid; idx < N * hw; idx += kRwWindow) {
            const int I = idx / hw, jl = idx - I * hw;
            int J = col0 - 1 + jl;
            J = J < 0 ? J + L : (J >= L ? J - L : J);
            word_st(win, (uint64_t)idx, word_ld<false>(S, (uint64_t)I * L + J, n_lat, __LINE__), n_win, __LINE__);
        }
    }
    if (PRE) {
        // the ring starts with the draws of steps 0 .. kRwRing - 1
        for (uint32_t j = tid; j < kRwRing && j < U; j += kRwWindow) ring_copy(&ring[j], &my_draws[j]);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    uint32_t next = 0;
    int cnt = 0, buf = 0;
    for (;;) {
        // the draws this round reads were copied at least three rounds ago
        // (a round takes at most kRwWindow steps and the ring holds
        // kRwRing = 4 kRwWindow), i.e. in groups older than the last two
        if (PRE) asm volatile("cp.async.wait_group 2;" ::: "memory");
        __syncthreads();
        // the free slots cnt .. take the next updates of the sequence
        const uint32_t fill = min((uint32_t)(kRwWindow - cnt), U - next);
        if (tid >= cnt && (uint32_t)(tid - cnt) < fill) {
            const uint32_t step = next + (uint32_t)(tid - cnt);
            uint32_t I, jr;
            uint64_t packed;
            if (PRE) {
                const ulonglong2 d = ring[step & (kRwRing - 1)];
                I = (uint32_t)d.x >> 16;
                jr = (uint32_t)d.x & 0xFFFFu;
                packed = d.y;
            } else {
                rw_draw(a, step, q, tl, x3, N, h, I, jr, packed);
            }
            sl_word[buf][tid] = I << 16 | jr;
            sl_mask[buf][tid] = packed;
        }
        next += fill;
        cnt += (int)fill;
        if (cnt == 0) break;
        __syncthreads();
        if (PRE) {
            // refill the ring positions just read with the draws kRwRing
            // steps on, which arrive while the next rounds run
            const uint32_t j = (uint32_t)tid;
            const uint32_t step = next - fill + kRwRing + j;
            if (j < fill && step < U) ring_copy(&ring[step & (kRwRing - 1)], &my_draws[step]);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // every pending update claims its word; the oldest claim wins
        const bool live = tid < cnt;
        uint32_t wI = 0, wj = 0, widx = 0;
        if (live) {
            const uint32_t word = sl_word[buf][tid];
            wI = word >> 16;
            wj = word & 0xFFFFu;
            widx = wI * (uint32_t)h + wj;
            atomicMin(&claim[widx & B], (uint32_t)tid);
        }
        __syncthreads();
        // it runs if no older pending update claims its word or a neighbour
        bool ready = false;
        if (live) {
            const uint32_t up = (wI == 0 ? (uint32_t)N - 1 : wI - 1) * (uint32_t)h + wj;
            const uint32_t dn = (wI == (uint32_t)N - 1 ? 0 : wI + 1) * (uint32_t)h + wj;
            ready = claim[widx & B] == (uint32_t)tid && claim[up & B] >= (uint32_t)tid &&
                    claim[dn & B] >= (uint32_t)tid;
            if (wj > 0) ready = ready && claim[(widx - 1) & B] >= (uint32_t)tid;
            if (wj + 1 < (uint32_t)h) ready = ready && claim[(widx + 1) & B] >= (uint32_t)tid;
        }
        __syncthreads();
        if (live) claim[widx & B] = 0xFFFFFFFFu;
        if (ready) {
            uint64_t s, xl, xr, xu, xd;
            uint64_t* dst;
            uint64_t didx, dn;
            if (WIN) {
                const uint64_t row = (uint64_t)wI * hw, jl = wj + 1;
                s = word_ld<false>(win, row + jl, n_win, __LINE__);
                xl = word_ld<false>(win, row + jl - 1, n_win, __LINE__);
                xr = word_ld<false>(win, row + jl + 1, n_win, __LINE__);
                xu = wI == 0 ? rotate_up(word_ld<false>(win, (uint64_t)(N - 1) * hw + jl, n_win, __LINE__))
                             : word_ld<false>(win, row - hw + jl, n_win, __LINE__);
                xd = wI == (uint32_t)N - 1 ? rotate_down(word_ld<false>(win, jl, n_win, __LINE__))
                                           : word_ld<false>(win, row + hw + jl, n_win, __LINE__);
                dst = win;
                didx = row + jl;
                dn = n_win;
            } else {
                const int J = col0 + (int)wj;
                const uint64_t row = (uint64_t)wI * L;
                s = word_ld<false>(S, row + J, n_lat, __LINE__);
                xl = word_ld<false>(S, row + (J == 0 ? L - 1 : J - 1), n_lat, __LINE__);
                xr = word_ld<false>(S, row + (J == L - 1 ? 0 : J + 1), n_lat, __LINE__);
                xu = wI == 0 ? rotate_up(word_ld<false>(S, (uint64_t)(N - 1) * L + J, n_lat, __LINE__))
                             : word_ld<false>(S, (uint64_t)(wI - 1) * L + J, n_lat, __LINE__);
                xd = wI == (uint32_t)N - 1 ? rotate_down(word_ld<false>(S, (uint64_t)J, n_lat, __LINE__))
                                           : word_ld<false>(S, (uint64_t)(wI + 1) * L + J, n_lat, __LINE__);
                dst = S;
                didx = row + J;
                dn = n_lat;
            }
            // Eq. 3: the 3-bit field sums hold a = 0..4 without carries
            const uint64_t A = (s ^ xu) + (s ^ xd) + (s ^ xl) + (s ^ xr);
            const uint64_t ge2 = ((A >> 1) | (A >> 2)) & kAllFields;
            const uint64_t any = (A | (A >> 1) | (A >> 2)) & kAllFields;
            const uint64_t m = sl_mask[buf][tid];
            const uint64_t c1 = (m & kAllFields) | all1, c0 = ((m >> 1) & kAllFields) | all0;
            const uint64_t accept = ge2 | (any & c1) | (~any & c0);
            word_st(dst, didx, s ^ (accept & kAllFields), dn, __LINE__);
        }
        __syncthreads();
        // the updates that did not run keep their order at the front
        const bool keep = live && !ready;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int lane = tid & 31, warp = tid >> 5;
        if (lane == 0) warp_keep[warp] = (uint32_t)__popc(bal);
        __syncthreads();
        int off = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kRwWindow / 32; ++k) {
            const int v = (int)warp_keep[k];
            off += k < warp ? v : 0;
            total += v;
        }
        if (keep) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            sl_word[buf ^ 1][pos] = sl_word[buf][tid];
            sl_mask[buf ^ 1][pos] = sl_mask[buf][tid];
        }
        buf ^= 1;
        cnt = total;
    }
    if (WIN) {
        // the half strip back to the lattice
        for (int idx = tid; idx < N * h; idx += kRwWindow) {
            const int I = idx / h, jr = idx - I * h;
            word_st(S, (uint64_t)I * L + col0 + jr, word_ld<false>(win, (uint64_t)I * hw + jr + 1, n_win, __LINE__),
                    n_lat, __LINE__);
        }
    }
}

// The apply-only half-sweep of the graph replays with one word per thread:
// thread k updates the colour-C word of word row I = k / (L / 2) in column
// pair m = k % (L / 2) with its masks from ci_mask_draw_kernel (`masks`: this
// sweep and colour's block, entry (q * L/2 + m) * 4 + e for I = 4q + e).  The
// spin logic is ci_half_sweep_kernel's; four times its threads, each with a
// quarter of the work, so a short half-sweep is not bound by the latency of
// a few threads' chains.  RECORD counts the colour-1 word's anti-aligned
// bonds and the up spins of both words of the column pair.
template <int C, bool RECORD>
__global__ void __launch_bounds__(128)
ci_half_sweep_apply_kernel(uint64_t* __restrict__ S, int L, int N, SweepArgs a, const uint64_t* __restrict__ masks)
{
    pdl_enter();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t half = (uint32_t)L / 2;
    uint32_t anti = 0, up = 0;
    if (k < (uint32_t)N * half) {
        const uint64_t n = (uint64_t)N * L;
        const int I = (int)(k / half), m = (int)(k - (uint32_t)I * half);
        const int J = 2 * m + ((I + C) & 1);
        const int Jl = J == 0 ? L - 1 : J - 1;
        const int Jr = J == L - 1 ? 0 : J + 1;
        const uint64_t row = (uint64_t)I * L;
        const uint64_t s = word_ld<false>(S, row + J, n, __LINE__);
        const uint64_t xl = word_ld<true>(S, row + Jl, n, __LINE__);
        const uint64_t xr = word_ld<true>(S, row + Jr, n, __LINE__);
        const uint64_t xu = I == 0 ? rotate_up(word_ld<true>(S, (uint64_t)(N - 1) * L + J, n, __LINE__))
                                   : word_ld<true>(S, (uint64_t)(I - 1) * L + J, n, __LINE__);
        const uint64_t xd = I == N - 1 ? rotate_down(word_ld<true>(S, (uint64_t)J, n, __LINE__))
                                       : word_ld<true>(S, (uint64_t)(I + 1) * L + J, n, __LINE__);
        const uint64_t packed = __ldg(masks + ((size_t)(I >> 2) * half + m) * 4 + (I & 3));
        const uint64_t all0 = ((uint64_t)a.all0 << 32 | a.all0) & kAllFields;
        const uint64_t all1 = ((uint64_t)a.all1 << 32 | a.all1) & kAllFields;
        // Eq. 3: each XOR field is 0/1, so the 3-bit sums hold a = 0..4 without carries
        const uint64_t A = (s ^ xu) + (s ^ xd) + (s ^ xl) + (s ^ xr);
        const uint64_t ge2 = ((A >> 1) | (A >> 2)) & kAllFields;
        const uint64_t any = (A | (A >> 1) | (A >> 2)) & kAllFields;
        const uint64_t accept = ge2 | (any & (packed | all1)) | (~any & ((packed >> 1) | all0));
        const uint64_t sn = s ^ (accept & kAllFields);
        word_st(S, row + J, sn, n, __LINE__);
        if (RECORD) {
            const uint64_t other = (J & 1) ? xl : xr;    // the other word of the column pair
            anti += __popcll(sn ^ xu) + __popcll(sn ^ xd) + __popcll(sn ^ xl) + __popcll(sn ^ xr);
            up += __popcll(sn) + __popcll(other);
        }
    }
    if (RECORD) block_add_counts(record_counts(a) + 2 * (blockIdx.x % kCountSlots), anti, up);
}

}  // namespace

bool ci_valid_side(int32_t L) { return L >= 84 && L <= 32760 && L % 84 == 0; }

bool ci_valid_strips(int32_t L, int32_t nstrips) { return nstrips >= 1 && L % nstrips == 0 && L / nstrips >= 2; }

size_t ci_rw_draw_bytes(int L, int nstrips)
{
    (void)nstrips;   // every strip draws 10 N per column: 10 N L updates per iteration
    return (size_t)10 * (L / 21) * L * sizeof(ulonglong2);
}

bool ci_rw_predraw(int L, int nstrips) { return ci_rw_draw_bytes(L, nstrips) <= kRwDrawBytesMax; }

cudaError_t ci_random_words_iteration(uint64_t* S, int L, int nstrips, const SweepArgs& a, ulonglong2* draws,
                                      cudaStream_t s)
{
    const int N = L / 21, NC = L / nstrips;
    const size_t win_bytes = (size_t)N * (NC - NC / 2 + 2) * sizeof(uint64_t);
    const bool win = win_bytes <= kRwWinBytesMax;
    static bool attr_set = false;   // per process; the attribute is per function
    if (win && !attr_set) {
        cudaError_t e = cudaFuncSetAttribute(ci_rw_phase_kernel<true, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRwWinBytesMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ci_rw_phase_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRwWinBytesMax);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const bool pre = draws != nullptr;
    if (pre) {
        const uint64_t total = 10ull * N * L;
        ci_rw_draw_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(L, N, NC, nstrips, a, draws);
    }
    for (int phase = 0; phase < 2; ++phase) {
        const int h = phase == 0 ? NC / 2 : NC - NC / 2;
        const size_t smem = win ? (size_t)N * (h + 2) * sizeof(uint64_t) : 0;
        const ulonglong2* d = pre ? draws + (phase ? (size_t)10 * N * (NC / 2) * nstrips : 0) : nullptr;
        if (pre && win) ci_rw_phase_kernel<true, true><<<nstrips, kRwWindow, smem, s>>>(S, L, N, NC, phase, a, d);
        else if (pre) ci_rw_phase_kernel<true, false><<<nstrips, kRwWindow, 0, s>>>(S, L, N, NC, phase, a, d);
        else if (win) ci_rw_phase_kernel<false, true><<<nstrips, kRwWindow, smem, s>>>(S, L, N, NC, phase, a, d);
        else ci_rw_phase_kernel<false, false><<<nstrips, kRwWindow, 0, s>>>(S, L, N, NC, phase, a, d);
    }
    return cudaGetLastError();
}

cudaError_t ci_init_hot(uint64_t* S, int L, uint64_t seed, cudaStream_t s)
{
    const int N = L / 21;
    dim3 block(32, 4);
    dim3 grid((L + 31) / 32, (N + 3) / 4);
    ci_init_hot_kernel<<<grid, block, 0, s>>>(S, L, N, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t ci_init_cold(uint64_t* S, int L, int up, cudaStream_t s)
{
    const size_t n = (size_t)(L / 21) * L;
    ci_fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S, n, up ? kAllFields : 0ull);
    return cudaGetLastError();
}

cudaError_t ci_pack(uint64_t* S, int L, const int8_t* spins, cudaStream_t s)
{
    const int N = L / 21;
    dim3 block(32, 4);
    dim3 grid((L + 31) / 32, (N + 3) / 4);
    ci_pack_kernel<<<grid, block, 0, s>>>(S, L, N, spins);
    return cudaGetLastError();
}

cudaError_t ci_unpack(const uint64_t* S, int L, int8_t* spins, cudaStream_t s)
{
    const int N = L / 21;
    dim3 block(32, 4);
    dim3 grid((L + 31) / 32, (N + 3) / 4);
    ci_unpack_kernel<<<grid, block, 0, s>>>(S, L, N, spins);
    return cudaGetLastError();
}

template <int ROUNDS>
static void ci_launch_r(dim3 grid, dim3 block, int colour, bool update, bool record, uint64_t* S, int L, int N,
                        const SweepArgs& a, cudaStream_t s)
{
    if (colour == 0) {
        if (record) ci_half_sweep_kernel<0, true, true, ROUNDS><<<grid, block, 0, s>>>(S, L, N, a, nullptr);
        else ci_half_sweep_kernel<0, true, false, ROUNDS><<<grid, block, 0, s>>>(S, L, N, a, nullptr);
    } else if (!update) {
        ci_half_sweep_kernel<1, false, true, 10><<<grid, block, 0, s>>>(S, L, N, a, nullptr);
    } else {
        if (record) ci_half_sweep_kernel<1, true, true, ROUNDS><<<grid, block, 0, s>>>(S, L, N, a, nullptr);
        else ci_half_sweep_kernel<1, true, false, ROUNDS><<<grid, block, 0, s>>>(S, L, N, a, nullptr);
    }
}

cudaError_t ci_half_sweep(int colour, bool update, bool record, uint64_t* S, int L, const SweepArgs& a,
                          cudaStream_t s)
{
    const int N = L / 21;
    dim3 block(32, 4);
    dim3 grid((L / 2 + 31) / 32, (N / 4 + 3) / 4);
    if (a.rounds == 7) ci_launch_r<7>(grid, block, colour, update, record, S, L, N, a, s);
    else ci_launch_r<10>(grid, block, colour, update, record, S, L, N, a, s);
    return cudaGetLastError();
}

size_t ci_mask_bytes_per_sweep(int L) { return (size_t)8 * (L / 21) * L; }

cudaError_t ci_mask_draw(int L, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                         uint64_t* masks, int blocks_per_sm, cudaStream_t s)
{
    const int N = L / 21;
    const long long threads = (long long)nsweeps * 2 * (N / 4) * (L / 2);
    unsigned blocks = (unsigned)((threads + 127) / 128);
    if (blocks_per_sm > 0) blocks = std::min(blocks, (unsigned)(device_sm_count() * blocks_per_sm));
    if (a.rounds == 7) ci_mask_draw_kernel<7><<<blocks, 128, 0, s>>>(L, N, a, t_base, t0, nsweeps, masks);
    else ci_mask_draw_kernel<10><<<blocks, 128, 0, s>>>(L, N, a, t_base, t0, nsweeps, masks);
    return cudaGetLastError();
}

cudaError_t ci_half_sweep_pre(int colour, bool record, uint64_t* S, int L, const SweepArgs& a,
                              const uint64_t* sweep_masks, cudaStream_t s)
{
    const int N = L / 21;
    const uint64_t* m = sweep_masks + (size_t)colour * (N / 4) * (L / 2) * 4;
    const unsigned threads = (unsigned)N * (unsigned)(L / 2);
    const dim3 grid((threads + 127) / 128), block(128);
    // programmatic dependent launch inside the graphs as for the row-packed
    // apply half-sweeps: up to 8192 and from 80000 thread items
    const int items = (N / 4) * (L / 2);
    const bool in_graphs = items <= 8192 || items >= 80000;
    if (colour == 0) launch_pdl_opt(in_graphs, ci_half_sweep_apply_kernel<0, false>, grid, block, s, S, L, N, a, m);
    else if (record) launch_pdl_opt(in_graphs, ci_half_sweep_apply_kernel<1, true>, grid, block, s, S, L, N, a, m);
    else launch_pdl_opt(in_graphs, ci_half_sweep_apply_kernel<1, false>, grid, block, s, S, L, N, a, m);
    return cudaGetLastError();
}

}  // namespace ising

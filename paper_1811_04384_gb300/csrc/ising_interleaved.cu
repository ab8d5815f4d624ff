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

namespace ising {
namespace {

constexpr uint64_t kAllFields = 0x1249249249249249ull;   // bit 3k, k = 0..20

__device__ __forceinline__ uint64_t rotate_up(uint64_t s)    // field k <- field k - 1 (periodic)
{
    return ((s << 3) | (s >> 60)) & kAllFields;
}

__device__ __forceinline__ uint64_t rotate_down(uint64_t s)  // field k <- field k + 1 (periodic)
{
    return ((s >> 3) | (s << 60)) & kAllFields;
}

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

// Accept masks of the words of thread (m, q) of ci_half_sweep_kernel for
// sweep t, colour C: Philox call k (counter (q + kN/4, m, t, C)) gives the
// draws of field k of the four words.  packed[e] holds r < thr1 of field k
// at bit 3k and r < thr0 at bit 3k + 1.
template <int ROUNDS>
__device__ __forceinline__ void ci_masks(int N, int q, int m, uint64_t t, int C, const SweepArgs& a,
                                         uint64_t packed[4])
{
    const uint32_t tl = (uint32_t)t;
    const uint32_t th = ((uint32_t)(t >> 32) << 1) | (uint32_t)C;
#pragma unroll
    for (int e = 0; e < 4; ++e) packed[e] = 0;
    for (int k = 0; k < 21; ++k) {
        const PhiloxRowKey pk = philox_row_key((uint32_t)(q + k * (N / 4)), tl, th, a.rk);
        uint32_t r[4];
        philox_row<ROUNDS>(pk, a.rk, (uint32_t)m, r);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            packed[e] |= (uint64_t)(r[e] < a.thr1) << (3 * k) | (uint64_t)(r[e] < a.thr0) << (3 * k + 1);
    }
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
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)nsweeps * 2 * Q * M) return;
    const int m = (int)(k % M);
    const int q = (int)((k / M) % Q);
    const int colour = (int)((k / (M * Q)) & 1);
    const int j = (int)(k / (2 * M * Q));
    uint64_t packed[4];
    ci_masks<ROUNDS>(N, q, m, (t_base ? *t_base : 0) + t0 + (uint64_t)j + 1, colour, a, packed);
#pragma unroll
    for (int e = 0; e < 4; ++e) masks[(size_t)k * 4 + e] = packed[e];
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
        uint64_t s[4], xl[4], xr[4], xu[4], xd[4], other[4];
        int J[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int I = 4 * q + e;
            J[e] = 2 * m + ((I + C) & 1);
            const int Jl = J[e] == 0 ? L - 1 : J[e] - 1;
            const int Jr = J[e] == L - 1 ? 0 : J[e] + 1;
            const uint64_t* row = S + (size_t)I * L;
            s[e] = row[J[e]];
            xl[e] = __ldg(row + Jl);
            xr[e] = __ldg(row + Jr);
            other[e] = (J[e] & 1) ? xl[e] : xr[e];    // the other word of the column pair
            xu[e] = I == 0 ? rotate_up(__ldg(S + (size_t)(N - 1) * L + J[e])) : __ldg(S + (size_t)(I - 1) * L + J[e]);
            xd[e] = I == N - 1 ? rotate_down(__ldg(S + J[e])) : __ldg(S + (size_t)(I + 1) * L + J[e]);
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
                S[(size_t)I * L + J[e]] = sn;
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

}  // namespace

bool ci_valid_side(int32_t L) { return L >= 84 && L <= 32760 && L % 84 == 0; }

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
                         uint64_t* masks, cudaStream_t s)
{
    const int N = L / 21;
    const long long threads = (long long)nsweeps * 2 * (N / 4) * (L / 2);
    const unsigned blocks = (unsigned)((threads + 127) / 128);
    if (a.rounds == 7) ci_mask_draw_kernel<7><<<blocks, 128, 0, s>>>(L, N, a, t_base, t0, nsweeps, masks);
    else ci_mask_draw_kernel<10><<<blocks, 128, 0, s>>>(L, N, a, t_base, t0, nsweeps, masks);
    return cudaGetLastError();
}

cudaError_t ci_half_sweep_pre(int colour, bool record, uint64_t* S, int L, const SweepArgs& a,
                              const uint64_t* sweep_masks, cudaStream_t s)
{
    const int N = L / 21;
    dim3 block(32, 4);
    dim3 grid((L / 2 + 31) / 32, (N / 4 + 3) / 4);
    const uint64_t* m = sweep_masks + (size_t)colour * (N / 4) * (L / 2) * 4;
    if (colour == 0) ci_half_sweep_kernel<0, true, false, 10, true><<<grid, block, 0, s>>>(S, L, N, a, m);
    else if (record) ci_half_sweep_kernel<1, true, true, 10, true><<<grid, block, 0, s>>>(S, L, N, a, m);
    else ci_half_sweep_kernel<1, true, false, 10, true><<<grid, block, 0, s>>>(S, L, N, a, m);
    return cudaGetLastError();
}

}  // namespace ising

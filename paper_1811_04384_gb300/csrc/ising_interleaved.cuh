// Device helpers of the paper's column-interleaved layout (Sec. 3, Fig. 1-2),
// shared by its kernels: the field rotations across the top and bottom word
// rows, and the accept masks of four words from the sites' own Philox draws.
#pragma once
#include <cstdint>

#include "ising_device.cuh"
#include "philox.cuh"

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

}  // namespace
}  // namespace ising

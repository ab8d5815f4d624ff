// Launchers of the paper's column-interleaved layout (ising_interleaved.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "ising_device.cuh"

namespace ising {

bool ci_valid_side(int32_t L);   // L % 84 == 0 (N = L / 21 divisible by 4), 84 <= L <= 32760
cudaError_t ci_init_hot(uint64_t* S, int L, uint64_t seed, cudaStream_t s);
cudaError_t ci_init_cold(uint64_t* S, int L, int up, cudaStream_t s);
cudaError_t ci_pack(uint64_t* S, int L, const int8_t* spins, cudaStream_t s);
cudaError_t ci_unpack(const uint64_t* S, int L, int8_t* spins, cudaStream_t s);
cudaError_t ci_half_sweep(int colour, bool update, bool record, uint64_t* S, int L, const SweepArgs& a,
                          cudaStream_t s);

}  // namespace ising

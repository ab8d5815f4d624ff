// Host-side helpers shared by the library's translation units (not part of
// the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "ising_device.cuh"

namespace ising {

// Record `e` with its call site for ising_last_cuda_error(); returns ISING_ECUDA.
int cuda_fail(cudaError_t e, const char* where);

// thr[a] = floor(2^32 exp(-(8 - 4a) beta)), clamped to [0, 2^32] (Sec. 2 step 3,
// Table 1), in IEEE double.
void thresholds_for_beta(double beta, uint64_t thr[2]);

// Kernel-argument form of the thresholds: clamped 32-bit values plus the
// "always accept" masks for a threshold of 2^32.
void fill_threshold_args(const uint64_t thr[2], SweepArgs& a);

Geom lattice_geom(int L);

cudaError_t launch_half_sweep(int rows, int bw, int bgrp, int colour, bool update, bool record,
                              uint64_t* own, const uint64_t* other, const Geom& g, const SweepArgs& a,
                              cudaStream_t s);

}  // namespace ising

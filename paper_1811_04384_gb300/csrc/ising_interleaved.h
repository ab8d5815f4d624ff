// Launchers of the paper's column-interleaved layout (ising_interleaved.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "ising_device.cuh"

namespace ising {

struct ClusterPlan;       // ising_internal.h
struct ClusterExchange;

bool ci_valid_side(int32_t L);   // L % 84 == 0 (N = L / 21 divisible by 4), 84 <= L <= 32760
cudaError_t ci_init_hot(uint64_t* S, int L, uint64_t seed, cudaStream_t s);
cudaError_t ci_init_cold(uint64_t* S, int L, int up, cudaStream_t s);
cudaError_t ci_pack(uint64_t* S, int L, const int8_t* spins, cudaStream_t s);
cudaError_t ci_unpack(const uint64_t* S, int L, int8_t* spins, cudaStream_t s);
cudaError_t ci_half_sweep(int colour, bool update, bool record, uint64_t* S, int L, const SweepArgs& a,
                          cudaStream_t s);
// Masks drawn ahead: ci_mask_draw fills `masks` with the accept masks of the
// nsweeps sweeps after sweep (t_base ? *t_base : 0) + t0 (both colours,
// ci_mask_bytes_per_sweep(L) bytes per sweep), with at most blocks_per_sm
// 128-thread blocks per SM (0: one thread per unit); ci_half_sweep_pre
// applies the block of one sweep (`sweep_masks`) to colour `colour`.
size_t ci_mask_bytes_per_sweep(int L);
cudaError_t ci_mask_draw(int L, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                         uint64_t* masks, int blocks_per_sm, cudaStream_t s);
cudaError_t ci_half_sweep_pre(int colour, bool record, uint64_t* S, int L, const SweepArgs& a,
                              const uint64_t* sweep_masks, cudaStream_t s);

// The paper's random-word chain (Sec. 4-5, Appendix A): iteration
// *a.t_base + a.t_off, phase 0 (the left floor(NC/2) columns of each of the
// nstrips strips of NC = L / nstrips columns) then phase 1 (the rest), one
// block per strip; thresholds and round keys from `a` (always 10 Philox
// rounds).  With `draws` (ci_rw_draw_bytes(L, nstrips) bytes of device
// memory; used when ci_rw_predraw(L, nstrips)) the updates' draws are made
// first on all SMs; with nullptr each block draws its own.
bool ci_valid_strips(int32_t L, int32_t nstrips);   // nstrips divides L, L / nstrips >= 2
size_t ci_rw_draw_bytes(int L, int nstrips);
// The cluster path in this layout (ising_ci_cluster.cu), as cluster_plan,
// cl_exchange_words, cl_mask_bytes_per_sweep, launch_cl_mask_draw and
// launch_cluster_sweeps of the row-packed one (ising_internal.h): the masks
// of nsweeps sweeps after sweep t0 (host value), then sweeps s0 + 1 ..
// s0 + nsweeps of a call.
bool ci_cluster_plan(int L, int clusters, ClusterPlan* plan);
size_t ci_cl_exchange_words(int L, const ClusterPlan& plan);
size_t ci_cl_mask_bytes_per_sweep(int L);
cudaError_t ci_cl_mask_draw(int L, const SweepArgs& a, uint64_t t0, int nsweeps, uint64_t* masks, bool overlap,
                            cudaStream_t s);
cudaError_t ci_cluster_sweeps(uint64_t* S, int L, const SweepArgs& a, const ClusterPlan& plan, int nsweeps,
                              const uint64_t* masks, int64_t s0, int64_t every, const ClusterExchange& x,
                              cudaStream_t s);
bool ci_rw_predraw(int L, int nstrips);
cudaError_t ci_random_words_iteration(uint64_t* S, int L, int nstrips, const SweepArgs& a, ulonglong2* draws,
                                      cudaStream_t s);

}  // namespace ising

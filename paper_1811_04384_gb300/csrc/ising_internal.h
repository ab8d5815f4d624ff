// Host-side helpers shared by the library's translation units (not part of
// the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>

#include "ising_device.cuh"

namespace ising {

// NVTX range for the duration of a scope (visible in Nsight timelines; a
// no-op unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Record `e` with its call site for ising_last_cuda_error(); returns ISING_ECUDA.
int cuda_fail(cudaError_t e, const char* where);

// thr[a] = floor(2^32 exp(-(8 - 4a) beta)), clamped to [0, 2^32] (Sec. 2 step 3,
// Table 1), in IEEE double.
void thresholds_for_beta(double beta, uint64_t thr[2]);

// Kernel-argument form of the thresholds: clamped 32-bit values plus the
// "always accept" masks for a threshold of 2^32.
void fill_threshold_args(const uint64_t thr[2], SweepArgs& a);

// Launch arguments for key `seed`, thresholds `thr`, device sweep counter
// t_base (t_off and counts left 0).
SweepArgs make_sweep_args(uint64_t seed, const uint64_t thr[2], const uint64_t* t_base);

Geom lattice_geom(int L);

// Launchers of the kernels in ising_kernels.cu (errors: the launch's own).
cudaError_t launch_init_hot(uint64_t* w0, uint64_t* w1, const Geom& g, uint64_t seed, cudaStream_t s);
cudaError_t launch_init_cold(uint64_t* w0, uint64_t* w1, const Geom& g, int up, cudaStream_t s);
cudaError_t launch_unpack(const uint64_t* w0, const uint64_t* w1, const Geom& g, int8_t* out, cudaStream_t s);
// int8 spins (row-major L x L, device memory or mapped pinned host memory) -> words.
cudaError_t launch_pack_rows(uint64_t* w0, uint64_t* w1, const Geom& g, const int8_t* src, cudaStream_t s);
// Device sweep counter: += n; += n with the graph record index += inc; = t.
cudaError_t launch_advance_sweep(uint64_t* t_base, uint64_t n, cudaStream_t s);
cudaError_t launch_advance_graph(uint64_t* t_base, uint64_t n, uint32_t* rec_base, uint32_t inc, cudaStream_t s);
cudaError_t launch_set_sweep(uint64_t* t_base, uint64_t t, cudaStream_t s);
// Philox4x32-10 of n counters (4 words each) under key `seed` (test hook).
cudaError_t launch_philox_blocks(const uint32_t* ctr, uint32_t* out, int64_t n, uint64_t seed, cudaStream_t s);
// The on-chip path: allow `bytes` of dynamic shared memory for its kernels
// (once), then run n sweeps from sweep t0 with one thread per item and E/M
// records every `every`-th sweep as (E, M) pairs into rec; `bytes` = both
// colour arrays.
cudaError_t allow_resident_smem(int bytes);
cudaError_t launch_resident(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a, uint64_t t0, int n,
                            int every, long long* rec, size_t bytes, cudaStream_t s);
// The on-chip path with masks drawn beforehand: draw the masks of the nsweeps
// sweeps after sweep (t_base ? *t_base : 0) + t0 (nsweeps * items * 4
// entries), then run sweeps s_base+1 ..
// s_base+n of a run reading them (at most kPremaskedMaxItems items, one or
// two rows per thread of one block; `bytes` = both colour arrays, and
// allow_resident_smem(bytes) leaves room for 1024 record counters).
constexpr int kPremaskedMaxItems = 512;
inline int premasked_rows_per_thread(int items) { return items <= 256 ? 1 : 2; }
// Two threads per row (one per 32-bit half of its word) up to 100 items: on
// GB300, 1000 recorded sweeps took 0.36 / 0.35 / 0.41 / 0.78 ms at L = 16 /
// 32 / 64 / 100 against 0.57 / 0.44 / 0.45 / 0.87 with one, but 0.99
// against 0.92 at L = 128 (128 items, 32 warps).
inline int premasked_threads_per_row(int items) { return items <= 100 ? 2 : 1; }
// blocks_per_sm > 0: at most that many 128-thread blocks per SM, each
// looping over its share (0: one thread per sweep and item).
cudaError_t launch_mask_draw(const Geom& g, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                             ulonglong2* masks, int blocks_per_sm, cudaStream_t s);
// SMs of the current device (1 if the query fails).
int device_sm_count();
// One half-sweep that applies masks drawn by launch_mask_draw (`masks`: the
// entries of its sweep), one thread per row.
cudaError_t launch_half_sweep_apply(int colour, bool record, uint64_t* own, const uint64_t* other, const Geom& g,
                                    const SweepArgs& a, const ulonglong2* masks, cudaStream_t s);
cudaError_t launch_resident_premasked(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a, int s_base,
                                      int n, int every, const ulonglong2* masks, long long* rec, size_t bytes,
                                      cudaStream_t s);

// The cluster path (ising_cluster.cu): one thread-block cluster whose blocks
// keep the lattice in their shared memory over many sweeps.  cluster_plan
// picks the launch for side L (false if there is none); launch_cl_mask_draw
// draws the masks of nsweeps sweeps after sweep (t_base ? *t_base : 0) + t0
// (cl_mask_bytes_per_sweep bytes each); with `overlap` it is launched with
// programmatic stream serialization, so that it runs beside the cluster
// launch before it in the stream (which must not read `masks`).
// launch_cluster_sweeps runs sweeps s0 + 1 .. s0 + nsweeps of a call from
// them, recording after every `every`-th (0: none) into count slot
// s / every - 1 past a.counts.
struct ClusterPlan {
    int blocks;     // cluster size
    int k;          // half-sweeps per phase = halo rows
    int q;          // mask slabs in shared memory
    int ns;         // window words per thread: 1 .. 4
    int threads;    // threads per block
    int clusters;   // clusters of a launch (1: the halos never leave the cluster)
};
// The rows crossing between the clusters of a launch (clusters > 1): `buf`
// holds cl_exchange_words(g, plan) words, `flags` 2 per cluster (zero when
// allocated, then only ever raised), `seq` the flag base of the launch (the
// caller adds cl_exchange_seqs(plan, nsweeps) after each launch), `err` a
// word set to 1 when a wait gave up, `wait_add` 0 (a test sets it to a value
// no push reaches, so that every wait of the launch gives up).
struct ClusterExchange {
    uint64_t* buf;
    unsigned long long* flags;
    unsigned long long seq;
    unsigned int* err;
    unsigned long long wait_add;   // added to the flag values a launch waits for (a test hook: nonzero stalls it)
    unsigned int* gate;            // the launch's agreement words (cl_count_in, cl_decide)
    unsigned int piece;            // the launch's piece of the call
    unsigned int absent;           // blocks counted on beyond the launch's (a test hook: 1 gives up)
};
bool cluster_plan(const Geom& g, int clusters, ClusterPlan* plan);
int cluster_max_active();   // clusters of one launch that can be resident at once (0: none)
size_t cl_exchange_words(const Geom& g, const ClusterPlan& plan);
unsigned long long cl_exchange_seqs(const ClusterPlan& plan, int nsweeps);
size_t cl_mask_bytes_per_sweep(const Geom& g);
cudaError_t launch_cl_mask_draw(const Geom& g, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                                uint64_t* masks, bool overlap, cudaStream_t s);
cudaError_t launch_cluster_sweeps(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a,
                                  const ClusterPlan& plan, int nsweeps, const uint64_t* masks, int64_t s0,
                                  int64_t every, const ClusterExchange& x, cudaStream_t s);

// Launch `kernel` with programmatic stream serialization (the kernel calls
// pdl_enter before its first read): the next launch's setup overlaps the end
// of the previous one.  On a stream that is being captured into a graph the
// launch is a plain one unless in_graphs: measured on GB300, programmatic
// edges made replayed graphs of the fused half-sweeps slower (L = 2016: 531
// -> 298 spin-updates/ns), while plain stream launches gained (L = 16384:
// +2.7%, L = 4096: +19%); the apply-only half-sweeps choose by size (see
// launch_half_sweep_apply).  Errors are left for cudaGetLastError.
template <typename... Params, typename... Args>
inline void launch_pdl_opt(bool in_graphs, void (*kernel)(Params...), dim3 grid, dim3 block, cudaStream_t s,
                           Args... args)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!in_graphs && cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... Params, typename... Args>
inline void launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, cudaStream_t s, Args... args)
{
    launch_pdl_opt(false, kernel, grid, block, s, args...);
}

// Geometry checks shared by the entry points.
bool valid_side(int32_t L);

// One half-sweep of one lattice (update and/or record), or the measurement
// pass (update = false, record = true, colour 1); block = bw x bgrp threads.
cudaError_t launch_half_sweep(int bw, int bgrp, int colour, bool update, bool record,
                              uint64_t* own, const uint64_t* other, const Geom& g, const SweepArgs& a,
                              cudaStream_t s);

// A half-sweep that updates, with F = 2, 4 or 8 lanes per thread item.
cudaError_t launch_half_sweep_lanes(int F, int colour, bool record, uint64_t* own, const uint64_t* other,
                                    const Geom& g, const SweepArgs& a, cudaStream_t s);

}  // namespace ising

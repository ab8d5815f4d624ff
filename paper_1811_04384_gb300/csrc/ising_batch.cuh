// The batched half-sweep: one launch per colour covers many replicas (used by
// the batch API and the server).
#pragma once
#include <cstdint>

#include "ising_device.cuh"

namespace ising {

// Device descriptor of one replica for the current run.
struct BatchReplica {
    uint64_t* w0;
    uint64_t* w1;
    Geom g;
    PhiloxKeys rk;
    uint32_t thr0, thr1, all0, all1;
    uint64_t t_start;               // sweep counter before this run
    uint32_t nsweeps;               // sweeps in this run
    uint32_t every;                 // record interval
    uint32_t phase;                 // records after sweeps s with (phase + s) % every == 0
    unsigned long long* counts;     // record k -> counts[2k], counts[2k+1] (anti, up)
    uint32_t items;                 // ceil(L/4) * W thread items
    uint32_t rounds;                // Philox rounds of the sweep draws (10 or the opt-in 7)
};

struct BatchTile {
    int rep;      // replica
    int first;    // first thread item of the tile
};

// One half-sweep of colour C over every replica that still has sweeps to do
// in this run.  Block b works on tile b; its threads own consecutive items
// item = group * W + w of the replica (4 rows x 1 word each).  ROUNDS: the
// Philox rounds of every replica (0: each replica's own, a runtime choice).
// REC: 0 records after the sweeps the replica's phase and interval pick, 1
// never records, 2 always records (colour 1).  Fixing both when a launch
// allows it removes the other code paths from the kernel: measured on GB300,
// scan 1,246 -> 1,284 and batched 1,262 -> 1,284 spin-updates/ns.
template <int C, int ROUNDS = 0, int REC = 0>
__global__ void __launch_bounds__(256, 3)
batch_half_sweep_kernel(const BatchReplica* __restrict__ reps, const BatchTile* __restrict__ tiles,
                        const uint32_t* __restrict__ chunk_base, uint32_t s_local, uint32_t one)
{
    pdl_enter();
    const BatchTile tile = tiles[blockIdx.x];
    const BatchReplica* R = reps + tile.rep;
    const uint32_t s = *chunk_base + s_local;      // sweep of this run, 1-based
    if (s > R->nsweeps) return;                    // uniform over the block
    const Geom g = R->g;
    const uint32_t item = (uint32_t)tile.first + threadIdx.x;
    const uint32_t ps = R->phase + s;
    const bool record = (C == 1) && (REC == 2 || (REC == 0 && ps % R->every == 0));
    uint32_t anti = 0, up = 0;
    if (item < R->items) {
        const int grp = (int)(item / (uint32_t)g.W);
        const int w = (int)(item - (uint32_t)grp * (uint32_t)g.W);
        const uint64_t t = R->t_start + s;
        uint64_t* own = C == 0 ? R->w0 : R->w1;
        const uint64_t* other = C == 0 ? R->w1 : R->w0;
        const PhiloxKeys rk = R->rk;
        const bool r7 = ROUNDS == 7 || (ROUNDS == 0 && R->rounds == 7);
        if (r7) {
            if (C == 1 && REC != 1 && record)
                sweep_rows<C, true, C == 1 && REC != 1, true, 7>(own, other, g, grp * 4, w, t, rk, R->thr0, R->thr1,
                                                                 R->all0, R->all1, one, anti, up);
            else if (REC != 2 || C == 0)
                sweep_rows<C, true, false, true, 7>(own, other, g, grp * 4, w, t, rk, R->thr0, R->thr1, R->all0,
                                                    R->all1, one, anti, up);
        } else if (ROUNDS != 7) {
            if (C == 1 && REC != 1 && record)
                sweep_rows<C, true, C == 1 && REC != 1>(own, other, g, grp * 4, w, t, rk, R->thr0, R->thr1, R->all0,
                                                        R->all1, one, anti, up);
            else if (REC != 2 || C == 0)
                sweep_rows<C, true, false>(own, other, g, grp * 4, w, t, rk, R->thr0, R->thr1, R->all0, R->all1,
                                           one, anti, up);
        }
    }
    if (record)
        block_add_counts(R->counts + 2 * (size_t)(ps / R->every - 1), anti, up);
}

static __global__ void batch_advance_kernel(uint32_t* chunk_base, uint32_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *chunk_base += n;
}

}  // namespace ising

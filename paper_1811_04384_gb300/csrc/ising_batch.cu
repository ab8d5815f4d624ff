// Batches of independent replicas (uneven L, own beta and seed) swept in
// lockstep: one kernel launch per colour covers every replica of a lane, its
// blocks being tiles of the replicas listed in a tile table; a chunk of
// sweeps is captured once into a CUDA graph and replayed.  The replicas are
// split into lanes of about equal work, and each lane is an independent
// branch of the graph, so the blocks of one lane fill the SMs that the last
// wave of another leaves idle.  Contract: include/ising.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "ising_internal.h"
#include "ising_batch.cuh"

using namespace ising;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxLanes = 8;
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct ising_batch {
    int n = 0;
    std::vector<Geom> geom;
    std::vector<double> beta;
    std::vector<uint64_t> seed;
    std::vector<uint64_t> t;                // host sweep counters
    std::vector<size_t> offset;             // byte offset of each replica's words in `arena`
    char* arena = nullptr;                  // all replicas' colour arrays
    BatchReplica* d_reps = nullptr;
    std::vector<BatchReplica> h_reps;
    BatchTile* d_tiles = nullptr;
    int ntiles = 0;
    int threads = 128;
    int chunk = 50;
    int lanes = 4;
    int lane_tile0[kMaxLanes] = {};         // first tile of each lane in d_tiles
    int lane_ntiles[kMaxLanes] = {};
    cudaStream_t lane_stream[kMaxLanes] = {};   // lane 0 runs on `stream`
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxLanes] = {};
    uint32_t* d_chunk_base = nullptr;
    unsigned long long* d_counts = nullptr;
    size_t counts_cap = 0;                  // in 64-bit words
    unsigned long long* h_counts = nullptr; // pinned mirror
    size_t h_counts_cap = 0;
    int8_t* staging = nullptr;
    size_t staging_cap = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;        // captured chunk of sweeps
    int graph_chunk = 0;
    int graph_threads = 0;
    int graph_lanes = 0;
    int graph_rounds = 0;                   // Philox rounds the graph's kernels are fixed for
    bool graph_every1 = false;              // colour-1 kernels record every sweep
};

namespace {

void free_batch(ising_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->arena);
    cudaFree(b->d_reps);
    cudaFree(b->d_tiles);
    cudaFree(b->d_chunk_base);
    cudaFree(b->d_counts);
    cudaFree(b->staging);
    if (b->h_counts) cudaFreeHost(b->h_counts);
    for (int k = 0; k < kMaxLanes; ++k) {
        if (b->lane_stream[k]) cudaStreamDestroy(b->lane_stream[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Lanes and tile table.  Replicas, largest first, go to the lane with the
// least work so far (L^2 each); each lane's tiles are contiguous in the
// table, every replica's items cut into blocks of `threads`.
int build_tiles(ising_batch* b)
{
    std::vector<int> order(b->n);
    for (int r = 0; r < b->n; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->geom[x].L > b->geom[y].L; });
    std::vector<int> lane_of(b->n, 0);
    double work[kMaxLanes] = {};
    for (int r : order) {
        int best = 0;
        for (int k = 1; k < b->lanes; ++k)
            if (work[k] < work[best]) best = k;
        lane_of[r] = best;
        work[best] += (double)b->geom[r].L * b->geom[r].L;
    }
    std::vector<BatchTile> tiles;
    for (int k = 0; k < kMaxLanes; ++k) {
        b->lane_tile0[k] = (int)tiles.size();
        for (int r : order) {
            if (k >= b->lanes || lane_of[r] != k) continue;
            const Geom& g = b->geom[r];
            const uint32_t items = (uint32_t)((g.L + 3) / 4) * (uint32_t)g.W;
            for (uint32_t f = 0; f < items; f += (uint32_t)b->threads) tiles.push_back({r, (int)f});
        }
        b->lane_ntiles[k] = (int)tiles.size() - b->lane_tile0[k];
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    cudaError_t e = cudaMalloc(&b->d_tiles, tiles.size() * sizeof(BatchTile));
    if (e != cudaSuccess) { cuda_fail(e, "cudaMalloc tiles"); return ISING_ENOMEM; }
    e = cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy tiles");
    b->ntiles = (int)tiles.size();
    return ISING_OK;
}

// Streams and events of lanes 1 .. lanes-1 (created once, kept).
int ensure_lane_streams(ising_batch* b)
{
    cudaError_t e = cudaSuccess;
    if (!b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 1; k < b->lanes && e == cudaSuccess; ++k) {
        if (!b->lane_stream[k]) e = cudaStreamCreateWithFlags(&b->lane_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b->join[k]) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "lane streams");
}

// Both half-sweeps of sweep s for one lane, with the kernel fixed for the
// batch-wide Philox rounds and, when every replica records every sweep,
// recording always.
template <int ROUNDS>
void launch_batch_pair_r(bool every1, dim3 grid, dim3 block, cudaStream_t st, const BatchReplica* reps,
                         const BatchTile* tiles, const uint32_t* chunk_base, uint32_t s)
{
    launch_pdl(batch_half_sweep_kernel<0, ROUNDS, 1>, grid, block, st, reps, tiles, chunk_base, s, 1u);
    if (every1) launch_pdl(batch_half_sweep_kernel<1, ROUNDS, 2>, grid, block, st, reps, tiles, chunk_base, s, 1u);
    else launch_pdl(batch_half_sweep_kernel<1, ROUNDS, 0>, grid, block, st, reps, tiles, chunk_base, s, 1u);
}

void launch_batch_pair(int rounds, bool every1, dim3 grid, dim3 block, cudaStream_t st, const BatchReplica* reps,
                       const BatchTile* tiles, const uint32_t* chunk_base, uint32_t s)
{
    if (rounds == 7) launch_batch_pair_r<7>(every1, grid, block, st, reps, tiles, chunk_base, s);
    else launch_batch_pair_r<10>(every1, grid, block, st, reps, tiles, chunk_base, s);
}

// One chunk of sweeps as a graph: lane 0 on the batch's stream, lanes
// 1.. forked from it and joined back before the chunk counter advances.
// The kernels are fixed for the batch's Philox rounds and for records every
// sweep, so the graph is recaptured when either changes.
int capture_graph(ising_batch* b, int rounds, bool every1)
{
    if (b->graph && b->graph_chunk == b->chunk && b->graph_threads == b->threads && b->graph_lanes == b->lanes &&
        b->graph_rounds == rounds && b->graph_every1 == every1)
        return ISING_OK;
    b->graph_rounds = rounds;
    b->graph_every1 = every1;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    int rc = ensure_lane_streams(b);
    if (rc != ISING_OK) return rc;
    cudaStream_t st[kMaxLanes];
    for (int k = 0; k < b->lanes; ++k) st[k] = k == 0 ? b->stream : b->lane_stream[k];
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t le = cudaEventRecord(b->fork, b->stream);
    for (int k = 1; k < b->lanes && le == cudaSuccess; ++k)
        if (b->lane_ntiles[k] > 0) le = cudaStreamWaitEvent(st[k], b->fork, 0);
    for (int s = 1; s <= b->chunk && le == cudaSuccess; ++s) {
        for (int k = 0; k < b->lanes && le == cudaSuccess; ++k) {
            const int nt = b->lane_ntiles[k];
            if (nt == 0) continue;
            const BatchTile* tiles = b->d_tiles + b->lane_tile0[k];
            launch_batch_pair(b->graph_rounds, b->graph_every1, dim3(nt), dim3(b->threads), st[k], b->d_reps, tiles,
                              b->d_chunk_base, (uint32_t)s);
            le = cudaGetLastError();
        }
    }
    for (int k = 1; k < b->lanes && le == cudaSuccess; ++k) {
        if (b->lane_ntiles[k] == 0) continue;
        le = cudaEventRecord(b->join[k], st[k]);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(b->stream, b->join[k], 0);
    }
    if (le == cudaSuccess) {
        batch_advance_kernel<<<1, 1, 0, b->stream>>>(b->d_chunk_base, (uint32_t)b->chunk);
        le = cudaGetLastError();
    }
    e = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(le, "batch capture launch"); }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    b->graph_chunk = b->chunk;
    b->graph_threads = b->threads;
    b->graph_lanes = b->lanes;
    return ISING_OK;
}

}  // namespace

extern "C" int ising_batch_create(int32_t n, const int32_t* L, const double* beta, const uint64_t* seed,
                                  const uint8_t* hot, ising_batch** out)
{
    if (!out || n < 1 || !L || !beta || !seed) return ISING_EINVAL;
    *out = nullptr;
    for (int r = 0; r < n; ++r) {
        if (!valid_side(L[r])) return ISING_EINVAL;
        if (std::isnan(beta[r]) || beta[r] < 0.0) return ISING_EINVAL;
    }
    ising_batch* b = new (std::nothrow) ising_batch();
    if (!b) return ISING_ENOMEM;
    b->n = n;
    size_t total = 0;
    for (int r = 0; r < n; ++r) {
        const Geom g = lattice_geom(L[r]);
        b->geom.push_back(g);
        b->beta.push_back(beta[r]);
        b->seed.push_back(seed[r]);
        b->t.push_back(0);
        b->offset.push_back(total);
        total += 2 * align_up((size_t)g.L * g.P * sizeof(uint64_t), kAlign);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { b->stream = nullptr; free_batch(b); return cuda_fail(e, "cudaStreamCreate"); }
    if (cudaMalloc(&b->arena, total) != cudaSuccess || cudaMalloc(&b->d_reps, n * sizeof(BatchReplica)) != cudaSuccess ||
        cudaMalloc(&b->d_chunk_base, sizeof(uint32_t)) != cudaSuccess) {
        free_batch(b);
        return ISING_ENOMEM;
    }
    e = cudaMemsetAsync(b->arena, 0, total, b->stream);
    for (int r = 0; r < n && e == cudaSuccess; ++r) {
        const Geom& g = b->geom[r];
        uint64_t* w0 = reinterpret_cast<uint64_t*>(b->arena + b->offset[r]);
        uint64_t* w1 = reinterpret_cast<uint64_t*>(b->arena + b->offset[r] + align_up((size_t)g.L * g.P * 8, kAlign));
        e = (hot && hot[r]) ? launch_init_hot(w0, w1, g, seed[r], b->stream) : launch_init_cold(w0, w1, g, 1, b->stream);
        BatchReplica R;
        std::memset(&R, 0, sizeof R);
        R.w0 = w0;
        R.w1 = w1;
        R.g = g;
        uint64_t thr[2];
        thresholds_for_beta(beta[r], thr);
        const SweepArgs a = make_sweep_args(seed[r], thr, nullptr);
        R.rk = a.rk;
        R.thr0 = a.thr0; R.thr1 = a.thr1; R.all0 = a.all0; R.all1 = a.all1;
        R.every = 1;
        R.rounds = 10;
        R.items = (uint32_t)((g.L + 3) / 4) * (uint32_t)g.W;
        b->h_reps.push_back(R);
    }
    if (e != cudaSuccess) { free_batch(b); return cuda_fail(e, "batch init"); }
    int rc = build_tiles(b);
    if (rc != ISING_OK) { free_batch(b); return rc; }
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { free_batch(b); return cuda_fail(e, "cudaStreamSynchronize"); }
    *out = b;
    return ISING_OK;
}

extern "C" int ising_batch_destroy(ising_batch* b)
{
    free_batch(b);
    return ISING_OK;
}

extern "C" int ising_batch_set_rng(ising_batch* b, int32_t scheme)
{
    if (!b) return ISING_EINVAL;
    uint32_t rounds;
    if (scheme == ISING_RNG_PHILOX4X32_10) rounds = 10;
    else if (scheme == ISING_RNG_PHILOX4X32_7) rounds = 7;
    else return ISING_EINVAL;
    for (BatchReplica& R : b->h_reps) R.rounds = rounds;
    return ISING_OK;
}

extern "C" int ising_batch_set_tiling(ising_batch* b, int32_t threads, int32_t chunk)
{
    if (!b) return ISING_EINVAL;
    if (threads != 64 && threads != 128 && threads != 256) return ISING_EINVAL;
    if (chunk < 1 || chunk > 1024) return ISING_EINVAL;
    const bool retile = threads != b->threads;
    b->threads = threads;
    b->chunk = chunk;
    if (retile) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        return build_tiles(b);
    }
    return ISING_OK;
}

extern "C" int ising_batch_set_lanes(ising_batch* b, int32_t lanes)
{
    if (!b || lanes < 1 || lanes > kMaxLanes) return ISING_EINVAL;
    if (lanes == b->lanes) return ISING_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    b->lanes = lanes;
    return build_tiles(b);
}

extern "C" int ising_batch_sweep(ising_batch* b, const int64_t* sweeps, int64_t every, int64_t** host_E,
                                 int64_t** host_M)
{
    TraceRange trace("ising_batch_sweep");
    if (!b || !sweeps || every < 1 || every > 0x7fffffff) return ISING_EINVAL;
    int64_t max_s = 0;
    size_t words = 0;
    std::vector<size_t> rec_off(b->n);
    for (int r = 0; r < b->n; ++r) {
        if (sweeps[r] < 0 || sweeps[r] > 0x7fffffff) return ISING_EINVAL;
        max_s = std::max(max_s, sweeps[r]);
        rec_off[r] = words;
        words += 2 * (size_t)(sweeps[r] / every);
    }
    if (max_s == 0) return ISING_OK;
    cudaError_t e;
    const size_t need = std::max<size_t>(words, 2);
    if (need > b->counts_cap) {
        cudaFree(b->d_counts);
        b->d_counts = nullptr;
        b->counts_cap = 0;
        e = cudaMalloc(&b->d_counts, need * sizeof(unsigned long long));
        if (e != cudaSuccess) { cuda_fail(e, "cudaMalloc counts"); return ISING_ENOMEM; }
        b->counts_cap = need;
    }
    if (need > b->h_counts_cap) {
        if (b->h_counts) cudaFreeHost(b->h_counts);
        b->h_counts = nullptr;
        b->h_counts_cap = 0;
        e = cudaMallocHost(&b->h_counts, need * sizeof(unsigned long long));
        if (e != cudaSuccess) { cuda_fail(e, "cudaMallocHost counts"); return ISING_ENOMEM; }
        b->h_counts_cap = need;
    }
    for (int r = 0; r < b->n; ++r) {
        BatchReplica& R = b->h_reps[r];
        R.t_start = b->t[r];
        R.nsweeps = (uint32_t)sweeps[r];
        R.every = (uint32_t)every;
        R.phase = 0;
        R.counts = b->d_counts + rec_off[r];
    }
    e = cudaMemcpyAsync(b->d_reps, b->h_reps.data(), b->n * sizeof(BatchReplica), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync replicas");
    e = cudaMemsetAsync(b->d_counts, 0, need * sizeof(unsigned long long), b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counts");
    e = cudaMemsetAsync(b->d_chunk_base, 0, sizeof(uint32_t), b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync chunk");
    int rc = capture_graph(b, b->h_reps[0].rounds == 7 ? 7 : 10, every == 1);
    if (rc != ISING_OK) return rc;
    const int64_t nlaunch = (max_s + b->chunk - 1) / b->chunk;
    for (int64_t k = 0; k < nlaunch; ++k) {
        e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    e = cudaMemcpyAsync(b->h_counts, b->d_counts, need * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync counts");
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int r = 0; r < b->n; ++r) {
        const int64_t N = (int64_t)b->geom[r].L * b->geom[r].L;
        const int64_t nrec = sweeps[r] / every;
        int64_t* E = host_E ? host_E[r] : nullptr;
        int64_t* M = host_M ? host_M[r] : nullptr;
        for (int64_t k = 0; k < nrec; ++k) {
            const unsigned long long* c = b->h_counts + rec_off[r] + 2 * k;
            if (E) E[k] = 2 * (int64_t)c[0] - 2 * N;
            if (M) M[k] = 2 * (int64_t)c[1] - N;
        }
        b->t[r] += (uint64_t)sweeps[r];
    }
    return ISING_OK;
}

extern "C" int ising_batch_get_spins(ising_batch* b, int32_t r, int8_t* out, size_t n)
{
    if (!b || !out || r < 0 || r >= b->n) return ISING_EINVAL;
    const Geom& g = b->geom[r];
    const size_t nn = (size_t)g.L * g.L;
    if (n != nn) return ISING_EINVAL;
    cudaError_t e;
    if (nn > b->staging_cap) {
        cudaFree(b->staging);
        b->staging = nullptr;
        b->staging_cap = 0;
        e = cudaMalloc(&b->staging, nn);
        if (e != cudaSuccess) { cuda_fail(e, "cudaMalloc staging"); return ISING_ENOMEM; }
        b->staging_cap = nn;
    }
    const BatchReplica& R = b->h_reps[r];
    e = launch_unpack(R.w0, R.w1, g, b->staging, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "unpack");
    e = cudaMemcpyAsync(out, b->staging, nn, cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync spins");
    e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "cudaStreamSynchronize");
}

extern "C" int ising_batch_get_sweep(ising_batch* b, int32_t r, uint64_t* t)
{
    if (!b || !t || r < 0 || r >= b->n) return ISING_EINVAL;
    *t = b->t[r];
    return ISING_OK;
}

extern "C" int ising_batch_run(int32_t n, const int32_t* L, const double* beta, const uint64_t* seed,
                               const uint8_t* hot, const int64_t* sweeps, int64_t every, int64_t** host_E,
                               int64_t** host_M, int8_t** final_spins)
{
    ising_batch* b = nullptr;
    int rc = ising_batch_create(n, L, beta, seed, hot, &b);
    if (rc != ISING_OK) return rc;
    rc = ising_batch_sweep(b, sweeps, every, host_E, host_M);
    for (int r = 0; rc == ISING_OK && final_spins && r < n; ++r)
        if (final_spins[r]) rc = ising_batch_get_spins(b, r, final_spins[r], (size_t)L[r] * L[r]);
    ising_batch_destroy(b);
    return rc;
}

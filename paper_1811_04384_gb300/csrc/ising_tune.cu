// Autotuner: times the launch shapes of the single-lattice path (and the
// on-chip path where the lattice fits) and the tile size / graph chunk /
// lanes of the batch path on the current device, checks that every candidate leaves a
// bit-identical lattice, and reports the fastest.  Contract: include/ising.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "../../include/ising.h"
#include "ising_internal.h"

namespace {

constexpr double kBetaTune = 1.0 / 2.269;   // timing point: the critical region (most uphill draws)
constexpr uint64_t kSeedTune = 0x5eed;

struct Candidate {
    int bw, bg, path, lanes;   // lanes per thread item on the launch path
};

// Time `sweeps` sweeps of a fresh hot-start lattice with candidate c; the
// final packed words go to *words.
int time_candidate(int32_t L, int32_t sweeps, const Candidate& c, double* ms, std::vector<uint64_t>* words)
{
    ising_lattice* h = nullptr;
    int rc = ising_create(L, kSeedTune, &h);
    if (rc != ISING_OK) return rc;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) rc = ising::cuda_fail(e, "autotune setup");
    if (rc == ISING_OK) rc = ising_set_stream(h, s);
    if (rc == ISING_OK) rc = ising_set_path(h, c.path);
    if (rc == ISING_OK && c.path == ISING_PATH_LAUNCHES) rc = ising_set_tiling(h, 4, c.bw, c.bg);
    if (rc == ISING_OK && c.path == ISING_PATH_LAUNCHES) rc = ising_set_item_lanes(h, c.lanes);
    if (rc == ISING_OK) rc = ising_init_hot(h);
    if (rc == ISING_OK) rc = ising_set_beta(h, kBetaTune);
    if (rc == ISING_OK) rc = ising_sweep(h, 33);                 // warm-up (module load, caches, graph capture)
    if (rc == ISING_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = ISING_ECUDA;
    if (rc == ISING_OK) rc = ising_sweep(h, sweeps);
    if (rc == ISING_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = ISING_ECUDA;
    if (rc == ISING_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = ISING_ECUDA;
    float f = 0.0f;
    if (rc == ISING_OK && cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) rc = ISING_ECUDA;
    *ms = f;
    if (rc == ISING_OK) {
        int32_t W = 0, P = 0, r = 0;
        ising_layout(h, &W, &P, &r);
        words->resize(2 * (size_t)L * P);
        rc = ising_get_words(h, words->data(), words->size());
    }
    ising_destroy(h);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}

}  // namespace

extern "C" int ising_autotune(int32_t L, int32_t sweeps, int32_t* best_bw, int32_t* best_bg, int32_t* best_path,
                              int32_t* best_lanes, double* ns_per_update)
{
    if (!ising::valid_side(L) || sweeps < 1 || sweeps > 100000) return ISING_EINVAL;
    const int P = ISING_PATH_LAUNCHES;
    std::vector<Candidate> cands = {{0, 128, P, 1},  {0, 64, P, 1},   {0, 192, P, 1},  {0, 256, P, 1},
                                    {32, 4, P, 1},   {16, 2, P, 1},   {16, 4, P, 1},   {16, 8, P, 1},
                                    {16, 16, P, 1},  {32, 1, P, 1},   {32, 2, P, 1},   {32, 8, P, 1},
                                    {64, 1, P, 1},   {64, 2, P, 1},   {64, 4, P, 1},   {0, 128, P, 2},
                                    {0, 128, P, 4},  {0, 128, P, 8},  {0, 128, ISING_PATH_RESIDENT, 0}};
    std::vector<uint64_t> ref, words;
    double best = -1.0;
    Candidate pick = cands[0];
    for (size_t k = 0; k < cands.size(); ++k) {
        double ms = 0.0;
        int rc = time_candidate(L, sweeps, cands[k], &ms, &words);
        if (rc == ISING_EINVAL && cands[k].path == ISING_PATH_RESIDENT) continue;   // does not fit on chip
        if (rc != ISING_OK) return rc;
        if (k == 0) ref = words;
        else if (words != ref) return ISING_ECUDA;     // a launch shape changed the results: never acceptable
        if (best < 0.0 || ms < best) {
            best = ms;
            pick = cands[k];
        }
    }
    if (best_bw) *best_bw = pick.bw;
    if (best_bg) *best_bg = pick.bg;
    if (best_path) *best_path = pick.path;
    if (best_lanes) *best_lanes = pick.lanes;
    if (ns_per_update) *ns_per_update = best * 1e6 / ((double)sweeps * L * L);
    return ISING_OK;
}

extern "C" int ising_batch_autotune(int32_t n, const int32_t* L, const double* beta, const uint64_t* seed,
                                    const uint8_t* hot, int64_t sweeps, int64_t every, int32_t* best_threads,
                                    int32_t* best_chunk, int32_t* best_lanes, double* ns_per_update)
{
    if (n < 1 || !L || !beta || !seed || sweeps < 1 || sweeps > 100000 || every < 1 || every > sweeps)
        return ISING_EINVAL;
    const int threads[3] = {64, 128, 256};
    const int chunks[3] = {10, 50, 200};
    const int lanes[3] = {1, 2, 4};
    double updates = 0.0;
    for (int r = 0; r < n; ++r) updates += (double)L[r] * L[r] * (double)sweeps;
    std::vector<int64_t> sw(n, sweeps);
    std::vector<std::vector<int8_t>> ref(n), got(n);
    double best = -1.0;
    int bt = 128, bc = 50, bl = 4;
    bool first = true;
    for (int ti = 0; ti < 3; ++ti) {
        for (int k = 0; k < 9; ++k) {
            const int ci = k % 3, li = k / 3;
            ising_batch* b = nullptr;
            int rc = ising_batch_create(n, L, beta, seed, hot, &b);
            if (rc != ISING_OK) return rc;
            rc = ising_batch_set_tiling(b, threads[ti], chunks[ci]);
            if (rc == ISING_OK) rc = ising_batch_set_lanes(b, lanes[li]);
            std::vector<int64_t> one(n, 1);
            if (rc == ISING_OK) rc = ising_batch_sweep(b, one.data(), every == 1 ? 1 : 2, nullptr, nullptr);   // warm-up
            // ising_batch_sweep synchronises the batch's stream, so the host clock times it
            const auto t0 = std::chrono::steady_clock::now();
            if (rc == ISING_OK) rc = ising_batch_sweep(b, sw.data(), every, nullptr, nullptr);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            for (int r = 0; rc == ISING_OK && r < n; ++r) {
                got[r].resize((size_t)L[r] * L[r]);
                rc = ising_batch_get_spins(b, r, got[r].data(), got[r].size());
            }
            ising_batch_destroy(b);
            if (rc != ISING_OK) return rc;
            if (first) ref = got;
            else if (got != ref) return ISING_ECUDA;
            first = false;
            if (best < 0.0 || ms < best) {
                best = ms;
                bt = threads[ti];
                bc = chunks[ci];
                bl = lanes[li];
            }
        }
    }
    if (best_threads) *best_threads = bt;
    if (best_chunk) *best_chunk = bc;
    if (best_lanes) *best_lanes = bl;
    if (ns_per_update) *ns_per_update = best * 1e6 / updates;
    return ISING_OK;
}

// ---- Integer pipe probe ---------------------------------------------------
// Throughput of the three integer instruction kinds the sweep is made of, in
// lane operations per SM per clock, read from the SM's own cycle counter (so
// it does not depend on the clock the GPU runs at): one block of 1024 threads
// per SM (its dynamic shared memory keeps a second block off the SM), each
// thread running kProbeChains independent dependency chains.
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeIters = 2048;
constexpr int kProbeThreads = 1024;
constexpr int kProbeSmem = 160 * 1024;

// KIND 0: the 32x32 -> 64-bit product of a Philox round (both halves);
// KIND 1: 32-bit multiply-add (low half only); KIND 2: three-input logic.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 1)
int_pipe_probe_kernel(uint32_t seed, uint32_t* sink, long long* cycles)
{
    extern __shared__ uint32_t probe_pad[];
    uint32_t x[kProbeChains], y[kProbeChains], z[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
        x[c] = seed ^ (threadIdx.x * kProbeChains + c);
        y[c] = x[c] * 0x9E3779B9u;
        z[c] = x[c] ^ 0xBB67AE85u;
    }
    if (threadIdx.x == 0) probe_pad[0] = seed;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            if (KIND == 0) {
                // the Philox round's product: both halves of M x, folded back
                // into x by an XOR (which issues on the other pipe)
                uint32_t hi, lo;
                ising::mul_hilo(ising::kPhiloxM0, x[c], hi, lo);
                x[c] = hi ^ lo;
            } else if (KIND == 1) {
                x[c] = x[c] * x[c] + y[c];           // a square: no two steps fold into one
            } else {
                // (x & y) ^ z: one three-input logic op, not linear, so no
                // sequence of steps simplifies into fewer; three steps per
                // iteration, each overwriting the oldest value, so that no
                // register moves are needed
                x[c] = (x[c] & y[c]) ^ z[c];
                y[c] = (y[c] & z[c]) ^ x[c];
                z[c] = (z[c] & x[c]) ^ y[c];
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t r = probe_pad[0];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) r ^= x[c] ^ y[c] ^ z[c];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = r;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
int run_probe(int nsm, uint32_t* sink, long long* d_cycles, double* rate)
{
    cudaError_t e = cudaFuncSetAttribute(int_pipe_probe_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kProbeSmem);
    if (e != cudaSuccess) return ising::cuda_fail(e, "probe attribute");
    for (int rep = 0; rep < 2; ++rep) {            // the first launch loads the module
        int_pipe_probe_kernel<KIND><<<nsm, kProbeThreads, kProbeSmem>>>(0x1234u + KIND, sink, d_cycles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return ising::cuda_fail(e, "int_pipe_probe_kernel");
    }
    std::vector<long long> cyc(nsm);
    e = cudaMemcpy(cyc.data(), d_cycles, nsm * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ising::cuda_fail(e, "probe cycles");
    std::sort(cyc.begin(), cyc.end());
    const double ops = (double)kProbeThreads * kProbeChains * kProbeIters * (KIND == 2 ? 3 : 1);
    *rate = cyc[nsm / 2] > 0 ? ops / (double)cyc[nsm / 2] : 0.0;
    return ISING_OK;
}

}  // namespace

extern "C" int ising_probe_int_pipes(double* mulwide_per_sm_clk, double* mad32_per_sm_clk, double* lop3_per_sm_clk,
                                     int32_t* sm_count)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ising::cuda_fail(e, "probe device");
    if (nsm < 1) return ISING_ECUDA;
    uint32_t* sink = nullptr;
    long long* d_cycles = nullptr;
    e = cudaMalloc(&sink, (size_t)nsm * kProbeThreads * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_cycles, (size_t)nsm * sizeof(long long));
    if (e != cudaSuccess) {
        cudaFree(sink);
        ising::cuda_fail(e, "cudaMalloc probe");
        return ISING_ENOMEM;
    }
    double r0 = 0, r1 = 0, r2 = 0;
    int rc = run_probe<0>(nsm, sink, d_cycles, &r0);
    if (rc == ISING_OK) rc = run_probe<1>(nsm, sink, d_cycles, &r1);
    if (rc == ISING_OK) rc = run_probe<2>(nsm, sink, d_cycles, &r2);
    cudaFree(sink);
    cudaFree(d_cycles);
    if (rc != ISING_OK) return rc;
    if (mulwide_per_sm_clk) *mulwide_per_sm_clk = r0;
    if (mad32_per_sm_clk) *mad32_per_sm_clk = r1;
    if (lop3_per_sm_clk) *lop3_per_sm_clk = r2;
    if (sm_count) *sm_count = nsm;
    return ISING_OK;
}

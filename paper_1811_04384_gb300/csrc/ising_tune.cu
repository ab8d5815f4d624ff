// Autotuner: times the launch shapes of the single-lattice path (and the
// on-chip path where the lattice fits) and the tile size / graph chunk /
// lanes of the batch path on the current device, checks that every candidate leaves a
// bit-identical lattice, and reports the fastest.  Contract: include/ising.h.
#include <cuda_runtime.h>

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

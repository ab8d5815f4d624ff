// Serving: continuous batching of simulation jobs on one device.  A worker
// thread admits queued jobs into a fixed device arena (first-fit), runs
// epochs of the batched half-sweep over every running job (split into lanes
// of about equal work on separate streams, so one lane's blocks fill the SMs
// another lane's last wave leaves idle), scatters each epoch's E/M records
// into the jobs' host arrays, and retires finished jobs.
// Contract: include/ising.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <stdexcept>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ising.h"
#include "ising_batch.cuh"
#include "ising_internal.h"

using namespace ising;

namespace {

constexpr size_t kAlign = 256;
constexpr int kLanes = 4;   // independent streams an epoch's jobs are split over
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

enum JobState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

// First-fit allocator over [0, capacity) with coalescing of free blocks.
class ArenaAllocator {
public:
    explicit ArenaAllocator(size_t capacity) : capacity_(capacity) { free_[0] = capacity; }
    bool alloc(size_t size, size_t* off)
    {
        size = align_up(size, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= size) {
                *off = it->first;
                const size_t rest = it->second - size;
                const size_t start = it->first + size;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t size)
    {
        size = align_up(size, kAlign);
        auto it = free_.emplace(off, size).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return capacity_; }

private:
    size_t capacity_;
    std::map<size_t, size_t> free_;
};

struct Job {
    ising_job spec;
    int state = kQueued;
    int status = ISING_EBUSY;
    double submit_s = 0, start_s = -1, done_s = -1;
    int64_t t = 0;                 // sweeps done
    size_t off = 0, bytes = 0;     // arena block
    Geom g;
    BatchReplica rep;
};

size_t job_bytes(int L)
{
    const Geom g = lattice_geom(L);
    return 2 * align_up((size_t)g.L * g.P * sizeof(uint64_t), kAlign);
}

}  // namespace

struct ising_server {
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable done_cv;  // wakes waiters
    std::unordered_map<uint64_t, Job> jobs;
    std::deque<uint64_t> queue;
    std::vector<uint64_t> running;
    uint64_t next_id = 1;
    bool stop = false;
    int device = 0;
    int max_jobs = 0;
    int epoch = 0;
    int fault_after = -1;             // test hook: epochs until an injected host exception (-1: none)
    std::chrono::steady_clock::time_point t0;
    // totals
    int64_t jobs_done = 0, epochs = 0;
    double updates = 0.0, busy_s = 0.0;
    // device state, owned by the worker
    ArenaAllocator* alloc = nullptr;
    char* arena = nullptr;
    BatchReplica* d_reps = nullptr;
    BatchTile* d_tiles = nullptr;
    size_t tiles_cap = 0;
    int ntiles = 0;
    uint32_t* d_zero = nullptr;
    unsigned long long* d_counts = nullptr;
    unsigned long long* h_counts = nullptr;
    int8_t* staging = nullptr;
    size_t staging_cap = 0;
    cudaStream_t stream = nullptr;                 // lane 0, copies
    cudaStream_t lane_stream[kLanes] = {};         // lanes 1 .. kLanes-1
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kLanes] = {};
    std::thread worker;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

int valid_job(const ising_job* j)
{
    if (!j || !valid_side(j->L)) return 0;
    if (std::isnan(j->beta) || j->beta < 0.0) return 0;
    if (j->sweeps < 1 || j->sweeps > 0x7fffffff || j->every < 1 || j->every > 0x7fffffff) return 0;
    if (j->rng != ISING_RNG_PHILOX4X32_10 && j->rng != ISING_RNG_PHILOX4X32_7) return 0;
    return 1;
}

// Mark every running job failed (after a device error or a host exception in
// the worker) and return its arena block, so that the queued jobs can still
// be admitted.
void fail_running(ising_server* s, int status)
{
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint64_t id : s->running) {
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) continue;
        Job& j = it->second;
        j.state = kFailed;
        j.status = status;
        j.done_s = s->now();
        s->alloc->release(j.off, j.bytes);
    }
    s->running.clear();
    s->done_cv.notify_all();
}

// Test hook (ising_server_inject_fault): throw a host exception at the start
// of the epoch the hook asked for, before any device work of that epoch.
void maybe_inject_fault(ising_server* s)
{
    bool fire = false;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->fault_after == 0) fire = true;
        if (s->fault_after >= 0) s->fault_after -= 1;
    }
    if (fire) throw std::runtime_error("injected server fault");
}

// Admit queued jobs in arrival order while a slot and arena space are free.
std::vector<uint64_t> admit(ising_server* s)
{
    std::vector<uint64_t> admitted;
    while (!s->queue.empty() && (int)s->running.size() < s->max_jobs) {
        const uint64_t id = s->queue.front();
        auto it = s->jobs.find(id);
        if (it == s->jobs.end() || it->second.state != kQueued) { s->queue.pop_front(); continue; }
        Job& j = it->second;
        size_t off;
        if (!s->alloc->alloc(j.bytes, &off)) break;
        s->queue.pop_front();
        j.off = off;
        j.state = kRunning;
        j.start_s = s->now();
        s->running.push_back(id);
        admitted.push_back(id);
    }
    return admitted;
}

int ensure_tiles(ising_server* s, size_t n)
{
    if (n <= s->tiles_cap) return ISING_OK;
    const size_t cap = std::max(n, 2 * s->tiles_cap);
    cudaFree(s->d_tiles);
    s->d_tiles = nullptr;
    s->tiles_cap = 0;
    cudaError_t e = cudaMalloc(&s->d_tiles, cap * sizeof(BatchTile));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc server tiles");
    s->tiles_cap = cap;
    return ISING_OK;
}

// One epoch over the running jobs (called by the worker without the lock; the
// running set and the jobs it names are only changed by the worker).
int run_epoch(ising_server* s, const std::vector<uint64_t>& run, std::vector<Job*>& jp)
{
    TraceRange trace("ising_server_epoch");
    const int threads = 128;
    std::vector<BatchReplica> reps(run.size());
    uint32_t max_n = 0;
    int rounds = 10;                               // 10 if every job uses Philox4x32-10, else per job
    std::vector<double> work(run.size());
    for (size_t a = 0; a < run.size(); ++a) {
        Job& j = *jp[a];
        BatchReplica& R = j.rep;
        const int64_t left = j.spec.sweeps - j.t;
        R.t_start = (uint64_t)j.t;
        R.nsweeps = (uint32_t)std::min<int64_t>(left, s->epoch);
        R.every = (uint32_t)j.spec.every;
        R.phase = (uint32_t)(j.t % j.spec.every);
        R.counts = s->d_counts + a * 2 * (size_t)s->epoch;
        reps[a] = R;
        max_n = std::max(max_n, R.nsweeps);
        if (R.rounds != 10) rounds = 0;
        work[a] = (double)j.g.L * j.g.L * R.nsweeps;
    }
    // lanes: jobs, most work first, to the lane with the least work so far;
    // each lane's tiles are contiguous and it runs on its own stream
    std::vector<size_t> order(run.size());
    for (size_t a = 0; a < order.size(); ++a) order[a] = a;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work[x] > work[y]; });
    std::vector<int> lane_of(run.size(), 0);
    double lane_work[kLanes] = {};
    for (size_t a : order) {
        int best = 0;
        for (int k = 1; k < kLanes; ++k)
            if (lane_work[k] < lane_work[best]) best = k;
        lane_of[a] = best;
        lane_work[best] += work[a];
    }
    std::vector<BatchTile> tiles;
    int lane_tile0[kLanes], lane_nt[kLanes];
    for (int k = 0; k < kLanes; ++k) {
        lane_tile0[k] = (int)tiles.size();
        for (size_t a : order)
            if (lane_of[a] == k)
                for (uint32_t f = 0; f < reps[a].items; f += threads) tiles.push_back({(int)a, (int)f});
        lane_nt[k] = (int)tiles.size() - lane_tile0[k];
    }
    int rc = ensure_tiles(s, tiles.size());
    if (rc != ISING_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(s->d_reps, reps.data(), reps.size() * sizeof(BatchReplica),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_counts, 0, run.size() * 2 * (size_t)s->epoch * sizeof(unsigned long long), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "server epoch setup");
    cudaStream_t st[kLanes];
    for (int k = 0; k < kLanes; ++k) st[k] = k == 0 ? s->stream : s->lane_stream[k];
    e = cudaEventRecord(s->fork, s->stream);
    for (int k = 1; k < kLanes && e == cudaSuccess; ++k)
        if (lane_nt[k] > 0) e = cudaStreamWaitEvent(st[k], s->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "server epoch fork");
    for (uint32_t n = 1; n <= max_n; ++n) {
        for (int k = 0; k < kLanes; ++k) {
            if (lane_nt[k] == 0) continue;
            const BatchTile* t = s->d_tiles + lane_tile0[k];
            const BatchReplica* R = s->d_reps;
            const uint32_t* z = s->d_zero;
            if (rounds == 10) {
                launch_pdl(batch_half_sweep_kernel<0, 10, 1>, dim3(lane_nt[k]), dim3(threads), st[k], R, t, z, n, 1u);
                launch_pdl(batch_half_sweep_kernel<1, 10, 0>, dim3(lane_nt[k]), dim3(threads), st[k], R, t, z, n, 1u);
            } else {
                launch_pdl(batch_half_sweep_kernel<0, 0, 1>, dim3(lane_nt[k]), dim3(threads), st[k], R, t, z, n, 1u);
                launch_pdl(batch_half_sweep_kernel<1, 0, 0>, dim3(lane_nt[k]), dim3(threads), st[k], R, t, z, n, 1u);
            }
        }
    }
    e = cudaGetLastError();
    for (int k = 1; k < kLanes && e == cudaSuccess; ++k) {
        if (lane_nt[k] == 0) continue;
        e = cudaEventRecord(s->join[k], st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->join[k], 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "server epoch launch");
    e = cudaMemcpyAsync(s->h_counts, s->d_counts, run.size() * 2 * (size_t)s->epoch * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "server epoch sync");
    // scatter the records, advance the jobs (under the lock: poll() reads t)
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t a = 0; a < run.size(); ++a) {
        Job& j = *jp[a];
        const BatchReplica& R = reps[a];
        const int64_t N = (int64_t)j.g.L * j.g.L;
        const int64_t nrec = (int64_t)(R.phase + R.nsweeps) / R.every;
        const int64_t base = j.t / j.spec.every;      // records before this epoch
        const unsigned long long* c = s->h_counts + a * 2 * (size_t)s->epoch;
        for (int64_t k = 0; k < nrec; ++k) {
            if (j.spec.host_E) j.spec.host_E[base + k] = 2 * (int64_t)c[2 * k] - 2 * N;
            if (j.spec.host_M) j.spec.host_M[base + k] = 2 * (int64_t)c[2 * k + 1] - N;
        }
        j.t += R.nsweeps;
        s->updates += (double)N * R.nsweeps;
    }
    return ISING_OK;
}

int copy_spins(ising_server* s, Job& j)
{
    const size_t nn = (size_t)j.g.L * j.g.L;
    cudaError_t e;
    if (nn > s->staging_cap) {
        cudaFree(s->staging);
        s->staging = nullptr;
        s->staging_cap = 0;
        e = cudaMalloc(&s->staging, nn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc server staging");
        s->staging_cap = nn;
    }
    e = launch_unpack(j.rep.w0, j.rep.w1, j.g, s->staging, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j.spec.host_spins, s->staging, nn, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "server spins");
}

// Wait for every stream of the server (used before failing the running jobs,
// so that no kernel still writes their arena blocks).
void drain_streams(ising_server* s)
{
    for (int k = 1; k < kLanes; ++k)
        if (s->lane_stream[k]) cudaStreamSynchronize(s->lane_stream[k]);
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaGetLastError();
}

void worker_main(ising_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<uint64_t> admitted, run;
        std::vector<Job*> jp;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait(lock, [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
            if (s->stop) break;
            admitted = admit(s);
            run = s->running;
            for (uint64_t id : run) jp.push_back(&s->jobs[id]);
        }
        if (run.empty()) {
            // the front job does not fit yet and nothing runs: cannot happen once
            // submit() rejects jobs larger than the arena; wait for news
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait_for(lock, std::chrono::milliseconds(5));
            continue;
        }
        try {
            // initialise the newly admitted jobs
            int rc = ISING_OK;
            for (uint64_t id : admitted) {
                Job* j = nullptr;
                {
                    std::lock_guard<std::mutex> lock(s->mu);
                    j = &s->jobs[id];
                }
                uint64_t* w0 = reinterpret_cast<uint64_t*>(s->arena + j->off);
                uint64_t* w1 = reinterpret_cast<uint64_t*>(s->arena + j->off + j->bytes / 2);
                cudaError_t e = cudaMemsetAsync(w0, 0, j->bytes, s->stream);
                if (e == cudaSuccess)
                    e = j->spec.hot ? launch_init_hot(w0, w1, j->g, j->spec.seed, s->stream)
                                    : launch_init_cold(w0, w1, j->g, 1, s->stream);
                if (e != cudaSuccess) { rc = cuda_fail(e, "server init"); break; }
                j->rep.w0 = w0;
                j->rep.w1 = w1;
            }
            const double t_begin = s->now();
            if (rc == ISING_OK) maybe_inject_fault(s);
            if (rc == ISING_OK) rc = run_epoch(s, run, jp);
            if (rc != ISING_OK) {
                fail_running(s, rc);
                continue;
            }
            // retire finished jobs
            std::vector<Job*> finished;
            for (Job* j : jp)
                if (j->t >= j->spec.sweeps) finished.push_back(j);
            for (Job* j : finished)
                j->status = j->spec.host_spins ? copy_spins(s, *j) : ISING_OK;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->busy_s += s->now() - t_begin;
                s->epochs += 1;
                for (Job* j : finished) {
                    j->state = j->status == ISING_OK ? kDone : kFailed;
                    j->done_s = s->now();
                    s->alloc->release(j->off, j->bytes);
                    s->jobs_done += 1;
                }
                s->running.erase(std::remove_if(s->running.begin(), s->running.end(),
                                                [&](uint64_t id) {
                                                    auto it = s->jobs.find(id);
                                                    return it == s->jobs.end() || it->second.state != kRunning;
                                                }),
                                 s->running.end());
                if (!finished.empty()) s->done_cv.notify_all();
            }
        } catch (...) {
            // A host exception in the worker (an allocation failure, or the
            // injected test fault): let the device finish what was launched,
            // fail the running jobs, and go on serving the queue.
            drain_streams(s);
            fail_running(s, ISING_EINTERNAL);
        }
    }
    // stopping: queued jobs are cancelled, running ones failed
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint64_t id : s->queue) {
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) continue;
        Job& j = it->second;
        if (j.state == kQueued) { j.state = kCancelled; j.status = ISING_EBUSY; }
    }
    for (uint64_t id : s->running) {
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) continue;
        Job& j = it->second;
        j.state = kFailed;
        j.status = ISING_EBUSY;
    }
    s->done_cv.notify_all();
}

void fill_result(const Job& j, ising_result* out)
{
    out->status = j.state == kDone ? ISING_OK : (j.state == kQueued || j.state == kRunning ? ISING_EBUSY : j.status);
    if (j.state == kCancelled) out->status = ISING_EBUSY;
    out->state = j.state;
    out->submit_s = j.submit_s;
    out->start_s = j.start_s;
    out->done_s = j.done_s;
    out->sweeps_done = j.t;
}

void free_server(ising_server* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->arena);
    cudaFree(s->d_reps);
    cudaFree(s->d_tiles);
    cudaFree(s->d_zero);
    cudaFree(s->d_counts);
    cudaFree(s->staging);
    if (s->h_counts) cudaFreeHost(s->h_counts);
    for (int k = 0; k < kLanes; ++k) {
        if (s->lane_stream[k]) cudaStreamDestroy(s->lane_stream[k]);
        if (s->join[k]) cudaEventDestroy(s->join[k]);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s->alloc;
    delete s;
}

}  // namespace

extern "C" int ising_server_create_ex(size_t budget, int32_t max_jobs, int32_t epoch_sweeps, ising_server** out)
{
    if (!out || budget < kAlign || max_jobs < 1 || max_jobs > 4096 || epoch_sweeps < 1 || epoch_sweeps > 100000)
        return ISING_EINVAL;
    if ((size_t)max_jobs * (size_t)epoch_sweeps > ((size_t)1 << 22)) return ISING_EINVAL;   // record buffer bound
    *out = nullptr;
    ising_server* s = new (std::nothrow) ising_server();
    if (!s) return ISING_ENOMEM;
    s->max_jobs = max_jobs;
    s->epoch = epoch_sweeps;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    budget = budget / kAlign * kAlign;
    s->alloc = new (std::nothrow) ArenaAllocator(budget);
    const size_t counts_words = (size_t)max_jobs * 2 * epoch_sweeps;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { s->stream = nullptr; free_server(s); return cuda_fail(e, "cudaStreamCreate"); }
    e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    for (int k = 1; k < kLanes && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->lane_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { free_server(s); return cuda_fail(e, "server lane streams"); }
    if (!s->alloc || cudaMalloc(&s->arena, budget) != cudaSuccess ||
        cudaMalloc(&s->d_reps, (size_t)max_jobs * sizeof(BatchReplica)) != cudaSuccess ||
        cudaMalloc(&s->d_zero, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&s->d_counts, counts_words * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&s->h_counts, counts_words * sizeof(unsigned long long)) != cudaSuccess) {
        free_server(s);
        return ISING_ENOMEM;
    }
    e = cudaMemset(s->d_zero, 0, sizeof(uint32_t));
    if (e != cudaSuccess) { free_server(s); return cuda_fail(e, "cudaMemset"); }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        free_server(s);
        return ISING_ENOMEM;
    }
    *out = s;
    return ISING_OK;
}

extern "C" int ising_server_create(size_t budget, ising_server** out)
{
    return ising_server_create_ex(budget, ISING_SERVER_DEFAULT_MAX_JOBS, ISING_SERVER_DEFAULT_EPOCH_SWEEPS, out);
}

extern "C" int ising_server_inject_fault(ising_server* s, int32_t epochs)
{
    if (!s || epochs < -1) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    s->fault_after = epochs;
    return ISING_OK;
}

extern "C" int ising_server_submit(ising_server* s, const ising_job* job, uint64_t* id)
{
    if (!s || !id || !valid_job(job)) return ISING_EINVAL;
    Job j;
    j.spec = *job;
    j.g = lattice_geom(job->L);
    j.bytes = job_bytes(job->L);
    if (j.bytes > s->alloc->capacity()) return ISING_ENOMEM;
    std::memset(&j.rep, 0, sizeof j.rep);
    j.rep.g = j.g;
    uint64_t thr[2];
    thresholds_for_beta(job->beta, thr);
    const SweepArgs a = make_sweep_args(job->seed, thr, nullptr);
    j.rep.rk = a.rk;
    j.rep.thr0 = a.thr0; j.rep.thr1 = a.thr1; j.rep.all0 = a.all0; j.rep.all1 = a.all1;
    j.rep.items = (uint32_t)((j.g.L + 3) / 4) * (uint32_t)j.g.W;
    j.rep.rounds = job->rng == ISING_RNG_PHILOX4X32_7 ? 7 : 10;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return ISING_EBUSY;
        j.submit_s = s->now();
        *id = s->next_id++;
        s->jobs.emplace(*id, j);
        s->queue.push_back(*id);
    }
    s->cv.notify_one();
    return ISING_OK;
}

extern "C" int ising_server_poll(ising_server* s, uint64_t id, ising_result* out)
{
    if (!s || !out) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return ISING_ENOTFOUND;
    fill_result(it->second, out);
    return ISING_OK;
}

extern "C" int ising_server_wait(ising_server* s, uint64_t id, int64_t timeout_ms, ising_result* out)
{
    if (!s || !out) return ISING_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto finished = [&] {
        auto it = s->jobs.find(id);
        return it == s->jobs.end() || (it->second.state != kQueued && it->second.state != kRunning);
    };
    if (timeout_ms < 0) s->done_cv.wait(lock, finished);
    else s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), finished);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return ISING_ENOTFOUND;
    fill_result(it->second, out);
    return finished() ? ISING_OK : ISING_ETIMEOUT;
}

extern "C" int ising_server_cancel(ising_server* s, uint64_t id)
{
    if (!s) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return ISING_ENOTFOUND;
    if (it->second.state != kQueued) return ISING_EBUSY;
    it->second.state = kCancelled;
    it->second.status = ISING_EBUSY;
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
    s->done_cv.notify_all();
    return ISING_OK;
}

extern "C" int ising_server_release(ising_server* s, uint64_t id)
{
    if (!s) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return ISING_ENOTFOUND;
    if (it->second.state == kQueued || it->second.state == kRunning) return ISING_EBUSY;
    s->jobs.erase(it);
    return ISING_OK;
}

extern "C" int ising_server_stats(ising_server* s, int64_t* jobs_done, double* updates, int64_t* epochs,
                                  double* busy_s)
{
    if (!s) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (jobs_done) *jobs_done = s->jobs_done;
    if (updates) *updates = s->updates;
    if (epochs) *epochs = s->epochs;
    if (busy_s) *busy_s = s->busy_s;
    return ISING_OK;
}

extern "C" int ising_server_destroy(ising_server* s)
{
    if (!s) return ISING_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    free_server(s);
    return ISING_OK;
}

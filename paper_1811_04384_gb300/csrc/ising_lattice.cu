// C ABI of the single-lattice path: handle management, initialisation,
// sweeps with the fused energy/magnetisation reduction (launches, graph
// replays, the on-chip path), spin I/O.  The kernels: ising_kernels.cu.
// Declarations and the contract of every function: include/ising.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "ising_device.cuh"
#include "ising_internal.h"
#include "ising_interleaved.h"

using namespace ising;

namespace {

constexpr int kRecordsPerChunk = 1024;           // count slots resident on the device
constexpr size_t kCountBytes = (size_t)kRecordsPerChunk * kCountSlots * 2 * sizeof(unsigned long long);
constexpr size_t kAlign = 256;
constexpr size_t kResidentMaxBytes = 220 * 1024;   // shared memory for the on-chip path
// auto: on-chip up to 128 thread items (L <= 128), the cluster path above;
// on a device without thread-block clusters on-chip up to 512 items (L <= 292).
// Measured on GB300 (sweeps without records / a record after every sweep,
// spin-updates/ns, on-chip against cluster): L = 100: 16.8 / 12.8 against
// 16.5 / 9.9; L = 128: 25.8 / 17.7 against 30.6 / 17.2; L = 168: 34.4 / 23.8
// against 55.8 / 31.0; L = 256: 27.8 / 22.8 against 102 / 59.
constexpr int kResidentAutoMaxItems = 128;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Geom make_geom(int L) { return lattice_geom(L); }

bool valid_L(int32_t L) { return valid_side(L); }

size_t words_bytes(const Geom& g) { return (size_t)g.L * (size_t)g.P * sizeof(uint64_t); }

}  // namespace

struct ising_lattice {
    Geom g;
    uint64_t seed = 0;
    uint64_t t = 0;              // host copy of the sweep counter
    double beta = 0.0;
    uint64_t thr[2] = {0, 0};
    cudaStream_t stream = nullptr;
    bool owns_mem = false;
    char* base = nullptr;        // device block: words0 | words1 | counts | t_base
    uint64_t* words[2] = {nullptr, nullptr};
    unsigned long long* counts = nullptr;
    uint64_t* t_dev = nullptr;
    int8_t* staging = nullptr;   // lazily allocated int8 L*L (get/set spins)
    int8_t* staging2 = nullptr;  // second input buffer of ising_run_states
    cudaStream_t copy_stream = nullptr;          // ising_run_states: host -> device copies
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_packed[2] = {nullptr, nullptr};
    unsigned long long* host_counts = nullptr;   // pinned, kCountBytes
    int bw = 0, bg = 128;                        // half-sweep shape: linear items, 128 threads a block
    int path = ISING_PATH_AUTO;                  // multi-block launches or on-chip resident sweeps
    int rounds = 10;                             // Philox rounds of the sweep draws
    int layout = ISING_LAYOUT_ROW_PACKED;        // or the paper's column-interleaved words
    int item_lanes = 0;                          // lanes per thread item on the launch path (0: auto)
    int chain = ISING_CHAIN_CHECKERBOARD;        // or the paper's random-word chain (interleaved layout)
    int nstrips = 1;                             // strips of the random-word chain
    ulonglong2* rw_draws = nullptr;              // random-word chain: the draws of one iteration (lazily)
    cudaStream_t capture_stream = nullptr;       // graphs of sweep chunks are captured here
    cudaGraphExec_t graph_plain = nullptr;       // kGraphSweeps sweeps, no record
    cudaGraphExec_t graph_rec = nullptr;         // record intervals of graph_rec_every sweeps, each recorded
    int graph_rec_every = 0;
    bool resident_attr = false;                  // dynamic shared memory attribute set
    ulonglong2* masks = nullptr;                 // lazily allocated: pre-drawn masks of the on-chip path
    size_t mask_bytes = 0;
    ulonglong2* graph_masks = nullptr;           // two buffers of draw_sweeps() sweeps' masks, drawn inside the graphs
    cudaStream_t draw_stream = nullptr;          // the graphs' mask draws are captured here, beside the half-sweeps
    cudaEvent_t fork_ev = nullptr, draw_ev[64] = {}, apply_ev[64] = {};   // kMaxPieces each
    int clusters = 0;                            // clusters of the cluster path's launches (0: automatic)
    uint64_t* xbuf = nullptr;                    // rows between clusters (lazily, several clusters only)
    size_t xbuf_bytes = 0;
    unsigned long long* xflag = nullptr;         // kXWords: their flags, the error word and the agreement words
    unsigned long long xseq = 0;                 // flag base of the next launch
    unsigned int* host_xerr = nullptr;           // pinned copy of the error and agreement words
    int stall_launches = 0;                      // test hook: launches whose waits between clusters give up
    int absent_after = -1;                       // test hook: the launch after this many more counts on one
                                                 // block more than it has (-1: none)
    bool multi_gave_up = false;                  // a launch's blocks were not all resident: auto keeps to one cluster
};

static void drop_graphs(ising_lattice* h);

extern "C" const char* ising_strerror(int code)
{
    switch (code) {
    case ISING_OK: return "ok";
    case ISING_EINVAL: return "invalid argument";
    case ISING_ENOMEM: return "out of memory";
    case ISING_ECUDA: return "CUDA error";
    case ISING_ETIMEOUT: return "timed out waiting";
    case ISING_EBUSY: return "busy: no free slot or memory budget";
    case ISING_ENOTFOUND: return "unknown request id";
    case ISING_EINTERNAL: return "internal host error in the server worker";
    default: return "unknown error code";
    }
}



extern "C" size_t ising_bytes_required(int32_t L)
{
    if (!valid_L(L)) return 0;
    const Geom g = make_geom(L);
    return 2 * align_up(words_bytes(g), kAlign) + align_up(kCountBytes, kAlign) + kAlign;
}

static int setup_handle(ising_lattice* h, int32_t L, uint64_t seed, char* base)
{
    h->g = make_geom(L);
    h->seed = seed;
    h->base = base;
    const size_t wb = align_up(words_bytes(h->g), kAlign);
    h->words[0] = reinterpret_cast<uint64_t*>(base);
    h->words[1] = reinterpret_cast<uint64_t*>(base + wb);
    h->counts = reinterpret_cast<unsigned long long*>(base + 2 * wb);
    h->t_dev = reinterpret_cast<uint64_t*>(base + 2 * wb + align_up(kCountBytes, kAlign));
    cudaError_t e = cudaMallocHost(&h->host_counts, kCountBytes);
    if (e != cudaSuccess) { h->host_counts = nullptr; return ISING_ENOMEM; }
    thresholds_for_beta(0.0, h->thr);
    return ISING_OK;
}

static void free_handle(ising_lattice* h)
{
    if (!h) return;
    if (h->rw_draws) cudaFree(h->rw_draws);
    if (h->staging) cudaFree(h->staging);
    if (h->staging2) cudaFree(h->staging2);
    if (h->masks) cudaFree(h->masks);
    if (h->graph_masks) cudaFree(h->graph_masks);
    if (h->xbuf) cudaFree(h->xbuf);
    if (h->xflag) cudaFree(h->xflag);
    if (h->host_xerr) cudaFreeHost(h->host_xerr);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
        if (h->ev_packed[b]) cudaEventDestroy(h->ev_packed[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->graph_plain) cudaGraphExecDestroy(h->graph_plain);
    if (h->graph_rec) cudaGraphExecDestroy(h->graph_rec);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->draw_stream) cudaStreamDestroy(h->draw_stream);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (cudaEvent_t ev : h->draw_ev) if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->apply_ev) if (ev) cudaEventDestroy(ev);
    if (h->owns_mem && h->base) cudaFree(h->base);
    if (h->host_counts) cudaFreeHost(h->host_counts);
    delete h;
}

extern "C" int ising_init_cold(ising_lattice* h, int8_t spin);

extern "C" int ising_create(int32_t L, uint64_t seed, ising_lattice** out)
{
    if (!out || !valid_L(L)) return ISING_EINVAL;
    *out = nullptr;
    ising_lattice* h = new (std::nothrow) ising_lattice();
    if (!h) return ISING_ENOMEM;
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, ising_bytes_required(L));
    if (e != cudaSuccess) { delete h; cuda_fail(e, "cudaMalloc"); return ISING_ENOMEM; }
    h->owns_mem = true;
    int rc = setup_handle(h, L, seed, base);
    if (rc == ISING_OK) rc = ising_init_cold(h, 1);
    if (rc != ISING_OK) { free_handle(h); return rc; }
    *out = h;
    return ISING_OK;
}

extern "C" int ising_create_layout(int32_t L, uint64_t seed, int32_t layout, ising_lattice** out)
{
    if (layout == ISING_LAYOUT_ROW_PACKED) return ising_create(L, seed, out);
    if (layout != ISING_LAYOUT_COLUMN_INTERLEAVED || !out || !ci_valid_side(L)) return ISING_EINVAL;
    *out = nullptr;
    ising_lattice* h = new (std::nothrow) ising_lattice();
    if (!h) return ISING_ENOMEM;
    // one N x L array of words, then the count slots and the sweep counter
    const size_t sb = align_up((size_t)(L / 21) * L * sizeof(uint64_t), kAlign);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, sb + align_up(kCountBytes, kAlign) + kAlign);
    if (e != cudaSuccess) { delete h; cuda_fail(e, "cudaMalloc"); return ISING_ENOMEM; }
    h->owns_mem = true;
    h->layout = layout;
    h->g = make_geom(L);
    h->seed = seed;
    h->base = base;
    h->words[0] = reinterpret_cast<uint64_t*>(base);
    h->words[1] = nullptr;
    h->counts = reinterpret_cast<unsigned long long*>(base + sb);
    h->t_dev = reinterpret_cast<uint64_t*>(base + sb + align_up(kCountBytes, kAlign));
    e = cudaMallocHost(&h->host_counts, kCountBytes);
    if (e != cudaSuccess) { h->host_counts = nullptr; free_handle(h); return ISING_ENOMEM; }
    thresholds_for_beta(0.0, h->thr);
    int rc = ising_init_cold(h, 1);
    if (rc != ISING_OK) { free_handle(h); return rc; }
    *out = h;
    return ISING_OK;
}

extern "C" int ising_create_on(int32_t L, uint64_t seed, void* dev_buf, size_t bytes, void* stream,
                               ising_lattice** out)
{
    if (!out || !valid_L(L) || !dev_buf) return ISING_EINVAL;
    if (bytes < ising_bytes_required(L) || ((uintptr_t)dev_buf % kAlign) != 0) return ISING_EINVAL;
    *out = nullptr;
    ising_lattice* h = new (std::nothrow) ising_lattice();
    if (!h) return ISING_ENOMEM;
    h->owns_mem = false;
    h->stream = (cudaStream_t)stream;
    int rc = setup_handle(h, L, seed, (char*)dev_buf);
    if (rc == ISING_OK) rc = ising_init_cold(h, 1);
    if (rc != ISING_OK) { free_handle(h); return rc; }
    *out = h;
    return ISING_OK;
}

extern "C" int ising_destroy(ising_lattice* h)
{
    if (!h) return ISING_OK;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    free_handle(h);
    return ISING_OK;
}

static int reset_t(ising_lattice* h, uint64_t t)
{
    cudaError_t e = launch_set_sweep(h->t_dev, t, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_sweep_kernel");
    h->t = t;
    return ISING_OK;
}

extern "C" int ising_init_hot(ising_lattice* h)
{
    TraceRange trace("ising_init_hot");
    if (!h) return ISING_EINVAL;
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED) {
        cudaError_t e = ci_init_hot(h->words[0], h->g.L, h->seed, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ci_init_hot");
        return reset_t(h, 0);
    }
    const Geom& g = h->g;
    // zero everything first so the pitch padding is defined
    cudaError_t e = cudaMemsetAsync(h->words[0], 0, 2 * align_up(words_bytes(g), kAlign), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = launch_init_hot(h->words[0], h->words[1], g, h->seed, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init_hot_kernel");
    return reset_t(h, 0);
}

extern "C" int ising_init_cold(ising_lattice* h, int8_t spin)
{
    if (!h || (spin != 1 && spin != -1)) return ISING_EINVAL;
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED) {
        cudaError_t e = ci_init_cold(h->words[0], h->g.L, spin > 0 ? 1 : 0, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ci_init_cold");
        return reset_t(h, 0);
    }
    cudaError_t e = launch_init_cold(h->words[0], h->words[1], h->g, spin > 0 ? 1 : 0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init_cold_kernel");
    return reset_t(h, 0);
}

extern "C" int ising_set_beta(ising_lattice* h, double beta)
{
    if (!h || std::isnan(beta) || beta < 0.0) return ISING_EINVAL;
    h->beta = beta;
    thresholds_for_beta(beta, h->thr);
    drop_graphs(h);                              // the thresholds are launch operands of the graphs
    return ISING_OK;
}

extern "C" int ising_get_thresholds(ising_lattice* h, uint64_t host_thr[2])
{
    if (!h || !host_thr) return ISING_EINVAL;
    host_thr[0] = h->thr[0];
    host_thr[1] = h->thr[1];
    return ISING_OK;
}

static SweepArgs base_args(const ising_lattice* h)
{
    SweepArgs a = make_sweep_args(h->seed, h->thr, h->t_dev);
    a.rounds = (uint32_t)h->rounds;
    return a;
}

// Lanes per thread item on the launch path: the handle's choice, else 4 up
// to 8192 items (L <= about 1100) and 1 above.  Measured on GB300 (sweeps
// without records, spin-updates/ns, F = 1 / 2 / 4 / 8 lanes): L = 512:
// 21 / 27 / 32 / 32; L = 1024: 85 / 102 / 128 / 128; L = 2048: 340 / 340 /
// 340 / 256; L = 4096: 815 / 680 / 584 / 454.  Below L = 2048 each launch is
// short and the lanes shorten it further; above, one thread per item fills
// the GPU and the merge is pure overhead.
static int item_lanes(const ising_lattice* h)
{
    if (h->item_lanes > 0) return h->item_lanes;
    const int items = ((h->g.L + 3) / 4) * h->g.W;
    return items <= 8192 ? 4 : 1;
}

// One half-sweep of the handle's lattice in its layout.
static cudaError_t launch_hs_on(const ising_lattice* h, cudaStream_t st, int colour, bool update, bool record,
                                const SweepArgs& a)
{
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED)
        return ci_half_sweep(colour, update, record, h->words[0], h->g.L, a, st);
    const int F = item_lanes(h);
    if (update && F > 1)
        return launch_half_sweep_lanes(F, colour, record, h->words[colour], h->words[1 - colour], h->g, a, st);
    return launch_half_sweep(h->bw, h->bg, colour, update, record, h->words[colour], h->words[1 - colour], h->g, a,
                             st);
}

static cudaError_t launch_hs(const ising_lattice* h, int colour, bool update, bool record, const SweepArgs& a)
{
    return launch_hs_on(h, h->stream, colour, update, record, a);
}

// ---- Graph replay of sweep chunks (launch path, small and mid-size lattices)
// Up to about L = 4100 (102400 thread items) the launch path runs chunks of
// sweeps as captured CUDA graphs: graph_plain holds kGraphSweeps sweeps, and
// graph_rec holds max(1, kGraphSweeps / every) record intervals of `every`
// sweeps, each recording into count slots offset by the device record index
// (advanced by the graph itself, so one graph serves every record of a
// chunk).  A graph draws the accept masks of draw_sweeps(h) sweeps at a time
// on all SMs (mask_draw_kernel, or ci_mask_draw in the column-interleaved
// layout, from the device sweep counter), and its half-sweeps only apply
// them (half_sweep_apply_kernel, ci_half_sweep_pre): at these sizes one
// thread per item leaves SMs idle while each runs its 21 Philox calls in a
// row, and a half-sweep runs about as long as the host takes to launch it.
// The draws run on a second branch of the graph, one piece ahead, into two
// alternating buffers: piece k + 1 is drawn while piece k is applied, and a
// piece is drawn into a buffer only after the half-sweeps of the piece before
// have read it.  The kernels' launch operands (thresholds, Philox rounds,
// launch shape) are baked into the graphs, so every call that changes them
// drops the graphs.  Measured on GB300, sweeps without records,
// spin-updates/ns, graphs against plain launches: L = 2600: 814 / 406;
// L = 3000: 889 / 575; L = 3500: 951 / 729; L = 4096: 996 / 966; but
// L = 4300: 1010 / 1082, where one thread per item fills the GPU.
constexpr int kGraphSweeps = 32;
constexpr int kGraphMaxEvery = 64;
constexpr int kGraphMaxItems = 102400;
constexpr int kMaxDrawSweeps = 8;
constexpr size_t kGraphMaskBytes = 32u << 20;    // both buffers
constexpr int kMaxPieces = kGraphMaxEvery;       // a graph holds at most kGraphMaxEvery sweeps

// Sweeps per drawn piece: 8, fewer where two buffers of 8 would pass 32 MB
// (64 B per item and sweep).
static int draw_sweeps(const ising_lattice* h)
{
    const size_t items = (size_t)((h->g.L + 3) / 4) * h->g.W;
    return (int)std::max<size_t>(1, std::min<size_t>(kMaxDrawSweeps, kGraphMaskBytes / (2 * 64 * items)));
}

// Blocks per SM of a graph's mask draws (0: one thread per unit): a capped
// grid whose blocks loop over the piece leaves room on every SM for the
// half-sweeps of the piece before, which run beside it on the other branch.
// Measured on GB300 (sweeps without records, spin-updates/ns, one thread per
// unit / 2 / 3 blocks per SM), row-packed: L = 1500: 508 / 539 / 532;
// L = 2016: 680 / 744 / 703; L = 3000: 887 / 941 / 915; L = 4096: 1006 / 923
// / 1035.  Column-interleaved: L = 1008: 305 / 283 / 291; L = 1512: 388 /
// 445 / 427; L = 2016: 511 / 575 / 552; L = 3024: 611 / 669 / 645;
// L = 4032: 683 / 295 / 360 (its half-sweeps use programmatic launches in the
// graphs from 80,000 items).
static int draw_blocks_per_sm(const ising_lattice* h)
{
    const int items = ((h->g.L + 3) / 4) * h->g.W;      // both layouts: the same thread count
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED) return items >= 10000 && items < 80000 ? 2 : 0;
    return items < 80000 ? 2 : 3;
}

static bool use_graphs(const ising_lattice* h)
{
    return ((h->g.L + 3) / 4) * h->g.W <= kGraphMaxItems;      // both layouts: the same thread count
}

static void drop_graphs(ising_lattice* h)
{
    if (h->graph_plain) cudaGraphExecDestroy(h->graph_plain);
    if (h->graph_rec) cudaGraphExecDestroy(h->graph_rec);
    h->graph_plain = nullptr;
    h->graph_rec = nullptr;
    h->graph_rec_every = 0;
}

static uint32_t* rec_index(const ising_lattice* h) { return reinterpret_cast<uint32_t*>(h->t_dev + 1); }

// Capture `n` sweeps (relative to the device counter) into *out.  every > 0:
// sweeps every, 2 every, ... record into the count slots 0, 1, ... past the
// device record index, which the graph then advances by n / every.
static int capture_sweeps(ising_lattice* h, int n, int every, cudaGraphExec_t* out)
{
    cudaError_t e = cudaSuccess;
    if (!h->capture_stream) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { h->capture_stream = nullptr; return cuda_fail(e, "capture stream"); }
    const bool ci = h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED;
    const size_t sweep_bytes = ci ? ci_mask_bytes_per_sweep(h->g.L)
                                  : (size_t)(((h->g.L + 3) / 4) * h->g.W) * 4 * sizeof(ulonglong2);
    const int D = draw_sweeps(h);
    if (!h->graph_masks) {
        e = cudaMalloc(&h->graph_masks, 2 * D * sweep_bytes);
        if (e != cudaSuccess) { h->graph_masks = nullptr; cuda_fail(e, "cudaMalloc graph masks"); return ISING_ENOMEM; }
    }
    if (!h->draw_stream) e = cudaStreamCreateWithFlags(&h->draw_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { h->draw_stream = nullptr; return cuda_fail(e, "draw stream"); }
    if (!h->fork_ev) e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < kMaxPieces && e == cudaSuccess; ++k) {
        if (!h->draw_ev[k]) e = cudaEventCreateWithFlags(&h->draw_ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->apply_ev[k]) e = cudaEventCreateWithFlags(&h->apply_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph events");
    SweepArgs a = base_args(h);
    cudaStream_t A = h->capture_stream;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(A, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    char* const buffers = reinterpret_cast<char*>(h->graph_masks);
    // one half-sweep of sweep s from its masks m (this sweep's block in a mask buffer)
    auto half = [&](int colour, bool rec, const char* m) {
        if (ci) return ci_half_sweep_pre(colour, rec, h->words[0], h->g.L, a, reinterpret_cast<const uint64_t*>(m), A);
        return launch_half_sweep_apply(colour, rec, h->words[colour], h->words[1 - colour], h->g, a,
                                       reinterpret_cast<const ulonglong2*>(m), A);
    };
    // the half-sweeps of sweep s (relative to the device counter)
    auto sweep = [&](int s, const char* m) {
        a.t_off = (uint32_t)s;
        a.counts = nullptr;
        a.rec_base = nullptr;
        cudaError_t r = half(0, false, m);
        const bool rec = every > 0 && s % every == 0;
        if (rec) {
            a.counts = h->counts + (size_t)(s / every - 1) * kCountSlots * 2;
            a.rec_base = rec_index(h);
        }
        if (r == cudaSuccess) r = half(1, rec, m);
        return r;
    };
    cudaStream_t B = h->draw_stream;
    const int np = (n + D - 1) / D;      // <= kMaxPieces
    auto draw = [&](int k) {       // piece k: sweeps k D + 1 .. into buffer k & 1
        const int first = k * D;
        const int count = std::min(D, n - first);
        char* buf = buffers + (size_t)(k & 1) * D * sweep_bytes;
        cudaError_t r = ci ? ci_mask_draw(h->g.L, a, h->t_dev, (uint64_t)first, count,
                                          reinterpret_cast<uint64_t*>(buf), draw_blocks_per_sm(h), B)
                           : launch_mask_draw(h->g, a, h->t_dev, (uint64_t)first, count,
                                              reinterpret_cast<ulonglong2*>(buf), draw_blocks_per_sm(h), B);
        if (r == cudaSuccess) r = cudaEventRecord(h->draw_ev[k], B);
        return r;
    };
    le = cudaEventRecord(h->fork_ev, A);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(B, h->fork_ev, 0);
    if (le == cudaSuccess) le = draw(0);
    for (int k = 0; k < np && le == cudaSuccess; ++k) {
        if (k + 1 < np) {
            if (k >= 1) le = cudaStreamWaitEvent(B, h->apply_ev[k - 1], 0);    // buffer (k + 1) & 1 is read
            if (le == cudaSuccess) le = draw(k + 1);
        }
        if (le == cudaSuccess) le = cudaStreamWaitEvent(A, h->draw_ev[k], 0);
        const char* buf = buffers + (size_t)(k & 1) * D * sweep_bytes;
        for (int s = k * D + 1; s <= std::min(n, (k + 1) * D) && le == cudaSuccess; ++s)
            le = sweep(s, buf + (size_t)(s - 1 - k * D) * sweep_bytes);
        if (le == cudaSuccess) le = cudaEventRecord(h->apply_ev[k], A);
    }
    if (le == cudaSuccess) {
        le = launch_advance_graph(h->t_dev, (uint64_t)n, rec_index(h), every > 0 ? (uint32_t)(n / every) : 0u, A);
    }
    e = cudaStreamEndCapture(A, &graph);
    if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(le, "sweep graph capture"); }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { *out = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return ISING_OK;
}

// n -> n % kGraphSweeps: the whole graph_plain chunks of n sweeps, replayed.
static int replay_plain(ising_lattice* h, int64_t* n)
{
    const int64_t reps = *n / kGraphSweeps;
    if (reps == 0) return ISING_OK;
    if (!h->graph_plain) {
        int rc = capture_sweeps(h, kGraphSweeps, 0, &h->graph_plain);
        if (rc != ISING_OK) return rc;
    }
    for (int64_t r = 0; r < reps; ++r) {
        cudaError_t e = cudaGraphLaunch(h->graph_plain, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    h->t += (uint64_t)(reps * kGraphSweeps);
    *n -= reps * kGraphSweeps;
    return ISING_OK;
}

// Run `n` sweeps relative to the device counter; sweep s (1-based) records into
// count slot rec_of(s) when rec_of(s) >= 0.  Then advances the counter by n.
template <typename RecOf>
static int run_sweeps(ising_lattice* h, int64_t n, RecOf rec_of)
{
    SweepArgs a = base_args(h);
    for (int64_t s = 1; s <= n; ++s) {
        a.t_off = (uint32_t)s;
        cudaError_t e = launch_hs(h, 0, true, false, a);
        if (e != cudaSuccess) return cuda_fail(e, "half_sweep colour 0");
        const int rec = rec_of(s);
        a.counts = rec >= 0 ? h->counts + (size_t)rec * kCountSlots * 2 : nullptr;
        e = launch_hs(h, 1, true, rec >= 0, a);
        if (e != cudaSuccess) return cuda_fail(e, "half_sweep colour 1");
    }
    if (n > 0) {
        cudaError_t e = launch_advance_sweep(h->t_dev, (uint64_t)n, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "advance_sweep_kernel");
        h->t += (uint64_t)n;
    }
    return ISING_OK;
}

// `records` x `every` sweeps, record r into count slots r: graph_rec holds
// per = max(1, kGraphSweeps / every) records; the records left over run as
// plain launches into their slots.
static int replay_records(ising_lattice* h, int64_t records, int every)
{
    const int per = std::max(1, kGraphSweeps / every);
    if (h->graph_rec && h->graph_rec_every != every) {
        cudaGraphExecDestroy(h->graph_rec);
        h->graph_rec = nullptr;
    }
    if (!h->graph_rec) {
        int rc = capture_sweeps(h, per * every, every, &h->graph_rec);
        if (rc != ISING_OK) return rc;
        h->graph_rec_every = every;
    }
    cudaError_t e = cudaMemsetAsync(rec_index(h), 0, sizeof(uint32_t), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync record index");
    const int64_t reps = records / per;
    for (int64_t r = 0; r < reps; ++r) {
        e = cudaGraphLaunch(h->graph_rec, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    h->t += (uint64_t)(reps * per * every);
    const int64_t done = reps * per, rest = records - done;
    if (rest == 0) return ISING_OK;
    return run_sweeps(h, rest * every, [every, done](int64_t s) {
        return (s % every == 0) ? (int)(done + s / every - 1) : -1;
    });
}


static size_t resident_bytes(const Geom& g) { return 2 * (size_t)g.L * g.P * sizeof(uint64_t); }

static bool use_resident(const ising_lattice* h)
{
    if (h->layout != ISING_LAYOUT_ROW_PACKED || (h->path != ISING_PATH_AUTO && h->path != ISING_PATH_RESIDENT))
        return false;
    if (resident_bytes(h->g) > kResidentMaxBytes) return false;
    if (h->path == ISING_PATH_RESIDENT) return true;
    const int items = ((h->g.L + 3) / 4) * h->g.W;
    if (items <= kResidentAutoMaxItems) return true;
    if (items > kPremaskedMaxItems) return false;
    ClusterPlan cp;
    return !cluster_plan(h->g, 1, &cp);
}

// Pre-drawn masks of the on-chip path: 64 B per item and sweep, drawn for
// at most this many bytes of sweeps at a time.
constexpr size_t kMaskBufMax = 16u << 20;

// n sweeps with the lattice resident in shared memory, E/M records (if any)
// written as (E, M) pairs into the count buffer.  Up to kPremaskedMaxItems
// items the accept masks are drawn first by all SMs (mask_draw_kernel), in
// pieces of at most kMaskBufMax bytes, and the on-chip kernel only applies
// them; larger lattices draw inside the on-chip kernel.
static int run_resident(ising_lattice* h, int n, int every)
{
    const Geom& g = h->g;
    if (!h->resident_attr) {
        cudaError_t e = allow_resident_smem((int)kResidentMaxBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        h->resident_attr = true;
    }
    const SweepArgs a = base_args(h);
    long long* rec = reinterpret_cast<long long*>(h->counts);
    const int items = ((g.L + 3) / 4) * g.W;
    if (items <= kPremaskedMaxItems) {
        const size_t per_sweep = (size_t)items * 4 * sizeof(ulonglong2);
        const int max_sweeps = (int)std::max<size_t>(1, kMaskBufMax / per_sweep);
        const size_t need = (size_t)std::min(n, max_sweeps) * per_sweep;
        if (h->mask_bytes < need) {
            if (h->masks) cudaFree(h->masks);
            h->masks = nullptr;
            h->mask_bytes = 0;
            cudaError_t e = cudaMalloc(&h->masks, need);
            if (e != cudaSuccess) { h->masks = nullptr; cuda_fail(e, "cudaMalloc masks"); return ISING_ENOMEM; }
            h->mask_bytes = need;
        }
        for (int done = 0; done < n;) {
            const int part = std::min(n - done, max_sweeps);
            cudaError_t e = launch_mask_draw(g, a, nullptr, h->t + (uint64_t)done, part, h->masks, 0, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "mask_draw_kernel");
            e = launch_resident_premasked(h->words[0], h->words[1], g, a, done, part, every, h->masks, rec,
                                          resident_bytes(g), h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "resident_premasked_kernel");
            done += part;
        }
    } else {
        cudaError_t e = launch_resident(h->words[0], h->words[1], g, a, h->t, n, every, rec, resident_bytes(g),
                                        h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "resident sweeps kernel");
    }
    cudaError_t e = launch_advance_sweep(h->t_dev, (uint64_t)n, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "advance_sweep_kernel");
    h->t += (uint64_t)n;
    return ISING_OK;
}

// ---- Cluster path (mid-size lattices)
// Above the on-chip range and up to kClusterMaxL, thread-block clusters keep
// the lattice in their blocks' shared memory over a whole piece of sweeps
// (cluster_sweeps_kernel): one cluster, or several (auto_clusters) whose
// boundary blocks pass their halo rows through a small global buffer.  The
// masks of each piece are drawn on all SMs into one of two buffers: the draw
// of piece j + 1 follows the cluster launch of piece j in the stream with
// programmatic stream serialization, so it runs on the SMs the clusters leave
// free while piece j is applied, and writes the buffer piece j - 1 read
// (complete before piece j started).  Replayed graphs of short half-sweeps
// stay for the launch path (ISING_PATH_LAUNCHES) and, above kClusterMaxL,
// the fused half-sweeps.  With one cluster (before several), sweeps without
// records, spin-updates/ns, cluster against graphs: L = 296: 138 / 34;
// L = 512: 255 / 96; L = 1008: 472 / 313; L = 1150: 499 / 362; but L = 1200:
// 297 / 368, where the window needs 4 words per thread, which spill
// registers.  Two 16 MB mask buffers (43-sweep pieces at L = 1008) gave 444
// there: each launch loads and writes back the lattice and refills the mask
// ring.  In the column-interleaved layout (one cluster): L = 1008: 373 /
// 304; L = 1092: 403 / 338; several clusters below (ci_auto_clusters).
constexpr int kClusterMaxL = 3000;
constexpr int kCiClusterMaxL = 2604;               // the column-interleaved layout (L % 84 == 0)
constexpr size_t kClusterMaskBytes = 256u << 20;   // both buffers
constexpr int kClusterMaxPiece = 256;
// The words between clusters (xflag, u64 each): 2 flags for each of at most
// 16 boundaries, the error word of the waits (u32), the agreement words
// (cl_decide: two sets of {count, verdict} and the first piece given up,
// u32 each); the host reads the status words [kXErr, kXWords) back.
constexpr int kXErr = 2 * 16;
constexpr int kXGate = kXErr + 1;
constexpr int kXWords = kXGate + 3;
constexpr int kXStatusWords = kXWords - kXErr;

// Clusters of a launch on the automatic path for side L (0: not the cluster
// path).  Measured on GB300, sweeps without records, spin-updates/ns by
// clusters 1 .. 7 (graph replays): L = 296: 124 / 86 / 73 / 55 / 29 / 28 / 27
// (34); L = 700: 302 / 352 / 383 / 381 / 347 / 300 / 300 (173); L = 1008:
// 439 / 506 / 552 / 667 / 638 / 626 / 598 (311); L = 1300: 240 / 651 / 717 /
// 739 / 767 / 773 / 723 (399); L = 1500: 409 / 771 / 922 / 904 / 943 / 904 /
// 880 (539); L = 2016: - / 657 / 993 / 1009 / 982 / 946 / 918 (742);
// L = 3000: four clusters 980 (939); L = 4096: seven 954 against the fused
// launches' 1031.  More clusters leave fewer SMs for the mask draws.
static int auto_clusters(int L)
{
    constexpr struct { int max_L, clusters; } kRule[] = {
        {558, 1}, {898, 3}, {1098, 4}, {1448, 6}, {1698, 5}, {kClusterMaxL, 4}};
    for (const auto& r : kRule)
        if (L <= r.max_L) return r.clusters;
    return 0;
}

// The same for the column-interleaved layout, whose per-word draws cost more
// (19 Philox products per call against 16), so the draws on the SMs the
// clusters leave free bound it sooner.  Measured on GB300, sweeps without
// records, spin-updates/ns by clusters 1 .. 7 (graph replays): L = 1008:
// 378 / 397 / 427 / 466 / 441 / 449 / 444 (305); L = 1512: 354 / 567 / 589 /
// 583 / 578 / 583 / 563 (444); L = 2016: - / 548 / 538 / 651 / 629 / 611 /
// 598 (574); L = 2520: three to seven 613 / 600 / 655 / 648 / 595 (633);
// L = 3024: four to seven 620 / 623 / 598 / 588 (666).
static int ci_auto_clusters(int L)
{
    constexpr struct { int max_L, clusters; } kRule[] = {
        {840, 1}, {1092, 4}, {1764, 3}, {2184, 4}, {kCiClusterMaxL, 5}};
    for (const auto& r : kRule)
        if (L <= r.max_L) return r.clusters;
    return 0;
}

static bool plan_cluster_g(const ising_lattice* h, int clusters, ClusterPlan* plan)
{
    return h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED ? ci_cluster_plan(h->g.L, clusters, plan)
                                                        : cluster_plan(h->g, clusters, plan);
}

static int auto_clusters_of(const ising_lattice* h)
{
    return h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED ? ci_auto_clusters(h->g.L) : auto_clusters(h->g.L);
}

// The cluster-path launch for h: the clusters set by ising_set_clusters, else
// the automatic count, or fewer where the device holds fewer clusters at
// once; one cluster on the automatic path once a launch found its blocks
// not all resident together (other work held SMs); `forced`
// (ISING_PATH_CLUSTER) also takes one cluster at any size it fits.
static bool plan_cluster(const ising_lattice* h, ClusterPlan* plan, bool forced)
{
    if (h->clusters > 0) return plan_cluster_g(h, h->clusters, plan);
    int G0 = auto_clusters_of(h);
    if (h->multi_gave_up && h->path == ISING_PATH_AUTO) G0 = std::min(G0, 1);
    for (int G = G0; G >= 1; --G)
        if (plan_cluster_g(h, G, plan)) return true;
    return forced && plan_cluster_g(h, 1, plan);
}

static bool use_cluster(const ising_lattice* h, ClusterPlan* plan)
{
    if (h->chain != ISING_CHAIN_CHECKERBOARD) return false;
    if (h->path == ISING_PATH_CLUSTER) return plan_cluster(h, plan, true);
    if (h->path != ISING_PATH_AUTO || use_resident(h)) return false;
    if (h->clusters == 0 && auto_clusters_of(h) == 0) return false;
    return plan_cluster(h, plan, false);
}

// n sweeps on the cluster path; every > 0: after every `every`-th sweep s of
// the n, a record into count slot s / every - 1 past `counts`.
static int run_cluster(ising_lattice* h, int64_t n, int64_t every, unsigned long long* counts, const ClusterPlan& plan)
{
    const Geom& g = h->g;
    const bool ci = h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED;
    const size_t per_sweep = ci ? ci_cl_mask_bytes_per_sweep(g.L) : cl_mask_bytes_per_sweep(g);
    const int max_piece =
        (int)std::max<size_t>(1, std::min<size_t>(kClusterMaxPiece, kClusterMaskBytes / (2 * per_sweep)));
    const size_t buf = (size_t)std::min<int64_t>(n, max_piece) * per_sweep;
    if (h->mask_bytes < 2 * buf) {
        if (h->masks) cudaFree(h->masks);
        h->masks = nullptr;
        h->mask_bytes = 0;
        cudaError_t e = cudaMalloc(&h->masks, 2 * buf);
        if (e != cudaSuccess) { h->masks = nullptr; cuda_fail(e, "cudaMalloc masks"); return ISING_ENOMEM; }
        h->mask_bytes = 2 * buf;
    }
    SweepArgs a = base_args(h);
    a.counts = counts;
    uint64_t* masks[2] = {reinterpret_cast<uint64_t*>(h->masks),
                          reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(h->masks) + buf)};
    // piece j: sweeps j * max_piece + 1 .. of the n, masks in buffer j & 1
    auto part_of = [&](int64_t j) { return (int)std::min<int64_t>(n - j * max_piece, max_piece); };
    const int64_t np = (n + max_piece - 1) / max_piece;
    auto draw = [&](int64_t j, bool overlap) {
        const uint64_t t0 = h->t + (uint64_t)(j * max_piece);
        return ci ? ci_cl_mask_draw(g.L, a, t0, part_of(j), masks[j & 1], overlap, h->stream)
                  : launch_cl_mask_draw(g, a, nullptr, t0, part_of(j), masks[j & 1], overlap, h->stream);
    };
    if (np > 0) {
        cudaError_t e = draw(0, false);
        if (e != cudaSuccess) return cuda_fail(e, "cluster mask draw");
    }
    ClusterExchange x = {nullptr, nullptr, 0, nullptr, 0, nullptr, 0, 0};
    const uint64_t t_start = h->t;
    if (plan.clusters > 1) {
        const size_t xb = (ci ? ci_cl_exchange_words(g.L, plan) : cl_exchange_words(g, plan)) * sizeof(uint64_t);
        cudaError_t e = cudaSuccess;
        if (h->xbuf_bytes < xb) {
            if (h->xbuf) cudaFree(h->xbuf);
            h->xbuf = nullptr;
            h->xbuf_bytes = 0;
            e = cudaMalloc(&h->xbuf, xb);
            if (e != cudaSuccess) { h->xbuf = nullptr; cuda_fail(e, "cudaMalloc exchange"); return ISING_ENOMEM; }
            h->xbuf_bytes = xb;
        }
        if (!h->xflag) {
            e = cudaMalloc(&h->xflag, kXWords * sizeof(unsigned long long));
            if (e == cudaSuccess) e = cudaMemsetAsync(h->xflag, 0, kXWords * sizeof(unsigned long long), h->stream);
            if (e == cudaSuccess && !h->host_xerr) e = cudaMallocHost(&h->host_xerr, kXStatusWords * sizeof(unsigned long long));
            if (e != cudaSuccess) { cuda_fail(e, "exchange flags"); return ISING_ENOMEM; }
            h->xseq = 0;
        }
        unsigned int* gate = reinterpret_cast<unsigned int*>(h->xflag + kXGate);
        // both agreement sets undecided, no piece given up
        e = cudaMemsetAsync(gate, 0, 4 * sizeof(unsigned int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(gate + 4, 0xff, sizeof(unsigned int), h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cluster agreement words");
        x = {h->xbuf, h->xflag, h->xseq, reinterpret_cast<unsigned int*>(h->xflag + kXErr), 0, gate, 0, 0};
    }
    for (int64_t j = 0; j < np; ++j) {
        const int64_t done = j * max_piece;
        x.wait_add = 0;
        x.piece = (unsigned int)j;
        x.absent = 0;
        if (plan.clusters > 1 && h->stall_launches > 0) {
            --h->stall_launches;
            x.wait_add = 1ull << 62;                 // no push reaches it: every wait gives up
        }
        if (plan.clusters > 1 && h->absent_after >= 0 && h->absent_after-- == 0)
            x.absent = 1;                            // one block more than the launch has: it gives up
        cudaError_t e = ci ? ci_cluster_sweeps(h->words[0], g.L, a, plan, part_of(j), masks[j & 1], done, every, x,
                                               h->stream)
                           : launch_cluster_sweeps(h->words[0], h->words[1], g, a, plan, part_of(j), masks[j & 1],
                                                   done, every, x, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cluster sweeps kernel");
        if (plan.clusters > 1) {
            x.seq += cl_exchange_seqs(plan, part_of(j));
            h->xseq = x.seq;
        }
        if (j + 1 < np) {
            e = draw(j + 1, true);
            if (e != cudaSuccess) return cuda_fail(e, "cluster mask draw");
        }
    }
    if (n > 0) {
        cudaError_t e = launch_advance_sweep(h->t_dev, (uint64_t)n, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "advance_sweep_kernel");
        h->t += (uint64_t)n;
    }
    if (plan.clusters > 1) {
        cudaError_t e = cudaMemcpyAsync(h->host_xerr, h->xflag + kXErr, kXStatusWords * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cluster exchange status");
        const unsigned int err = h->host_xerr[0];
        const unsigned int gave_up = h->host_xerr[2 * (kXGate - kXErr) + 4];
        if (err != 0) {
            e = cudaMemsetAsync(x.err, 0, sizeof(unsigned int), h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cluster exchange status");
            h->host_xerr[0] = 0;
        }
        if (gave_up != 0xffffffffu) {
            // the launch of piece gave_up did not have all its blocks resident
            // together: it wrote no lattice row, nor did the launches after
            // it.  The pieces before it stand; its records are cleared and the
            // rest of the call runs on the launch path (the same draws, so the
            // same results); the automatic path keeps to one cluster from now on.
            const int64_t done = (int64_t)gave_up * max_piece;
            h->multi_gave_up = true;
            int rc = reset_t(h, t_start + (uint64_t)done);
            if (rc != ISING_OK) return rc;
            const int64_t rec_base = (int64_t)(counts - h->counts) / (2 * kCountSlots);
            if (every > 0 && n / every > done / every) {
                const size_t slot_bytes = 2 * kCountSlots * sizeof(unsigned long long);
                e = cudaMemsetAsync(counts + (size_t)(done / every) * 2 * kCountSlots, 0,
                                    (size_t)(n / every - done / every) * slot_bytes, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cluster records");
            }
            return run_sweeps(h, n - done, [every, done, rec_base](int64_t s) {
                return (every > 0 && (done + s) % every == 0) ? (int)(rec_base + (done + s) / every - 1) : -1;
            });
        }
        // a wait between clusters that gave up while all were resident voids
        // the sweeps (the counter has advanced; the caller restores a
        // checkpoint to retry)
        if (err != 0) return ISING_ETIMEOUT;
    }
    return ISING_OK;
}

extern "C" int ising_set_clusters(ising_lattice* h, int32_t clusters)
{
    if (!h || clusters < 0 || clusters > 16) return ISING_EINVAL;
    ClusterPlan cp;
    if (clusters > 0 && !plan_cluster_g(h, clusters, &cp)) return ISING_EINVAL;
    h->clusters = clusters;
    h->multi_gave_up = false;
    return ISING_OK;
}

extern "C" int ising_cluster_inject_stall(ising_lattice* h, int32_t launches)
{
    if (!h || launches < 0) return ISING_EINVAL;
    h->stall_launches = launches;
    return ISING_OK;
}

extern "C" int ising_cluster_inject_absent(ising_lattice* h, int32_t after)
{
    if (!h || after < -1) return ISING_EINVAL;
    h->absent_after = after;
    return ISING_OK;
}

extern "C" int ising_set_rng(ising_lattice* h, int32_t scheme)
{
    if (!h) return ISING_EINVAL;
    if (scheme == ISING_RNG_PHILOX4X32_10) h->rounds = 10;
    else if (scheme == ISING_RNG_PHILOX4X32_7) h->rounds = 7;
    else return ISING_EINVAL;
    drop_graphs(h);
    return ISING_OK;
}

extern "C" int ising_set_path(ising_lattice* h, int32_t path)
{
    if (!h) return ISING_EINVAL;
    if (path != ISING_PATH_AUTO && path != ISING_PATH_LAUNCHES && path != ISING_PATH_RESIDENT &&
        path != ISING_PATH_CLUSTER)
        return ISING_EINVAL;
    if (path == ISING_PATH_RESIDENT && (h->layout != ISING_LAYOUT_ROW_PACKED || resident_bytes(h->g) > kResidentMaxBytes))
        return ISING_EINVAL;
    ClusterPlan cp;
    if (path == ISING_PATH_CLUSTER && !plan_cluster(h, &cp, true)) return ISING_EINVAL;
    h->path = path;
    h->multi_gave_up = false;
    return ISING_OK;
}

extern "C" int ising_get_path(ising_lattice* h, int32_t* path)
{
    if (!h || !path) return ISING_EINVAL;
    ClusterPlan cp;
    if (h->chain == ISING_CHAIN_RANDOM_WORDS) *path = h->path;
    else if (use_resident(h)) *path = ISING_PATH_RESIDENT;
    else if (use_cluster(h, &cp)) *path = ISING_PATH_CLUSTER;
    else *path = ISING_PATH_LAUNCHES;
    return ISING_OK;
}

// The paper's random-word chain: iterations t+1 .. t+n (relative to the
// device counter), each its two phases; iteration s (1-based) is followed by
// an E/M measurement into count slot rec_of(s) when rec_of(s) >= 0.
template <typename RecOf>
static int run_random_words(ising_lattice* h, int64_t n, RecOf rec_of)
{
    SweepArgs a = base_args(h);
    // the updates' draws are made first on all SMs unless the launch path was
    // chosen or the buffer would be too large; then each block draws its own
    const bool pre = h->path != ISING_PATH_LAUNCHES && ci_rw_predraw(h->g.L, h->nstrips);
    if (pre && !h->rw_draws) {
        cudaError_t e = cudaMalloc(&h->rw_draws, ci_rw_draw_bytes(h->g.L, h->nstrips));
        if (e != cudaSuccess) { h->rw_draws = nullptr; cuda_fail(e, "cudaMalloc random-word draws"); return ISING_ENOMEM; }
    }
    for (int64_t it = 1; it <= n; ++it) {
        a.t_off = (uint32_t)it;
        a.counts = nullptr;
        cudaError_t e = ci_random_words_iteration(h->words[0], h->g.L, h->nstrips, a, pre ? h->rw_draws : nullptr,
                                                  h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ci_rw_phase_kernel");
        const int rec = rec_of(it);
        if (rec >= 0) {
            a.counts = h->counts + (size_t)rec * kCountSlots * 2;
            cudaError_t e = ci_half_sweep(1, false, true, h->words[0], h->g.L, a, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "measure");
        }
    }
    if (n > 0) {
        cudaError_t e = launch_advance_sweep(h->t_dev, (uint64_t)n, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "advance_sweep_kernel");
        h->t += (uint64_t)n;
    }
    return ISING_OK;
}

extern "C" int ising_set_chain(ising_lattice* h, int32_t chain, int32_t nstrips)
{
    if (!h) return ISING_EINVAL;
    if (chain == ISING_CHAIN_CHECKERBOARD) {
        h->chain = chain;
        h->nstrips = 1;
        return ISING_OK;
    }
    if (chain != ISING_CHAIN_RANDOM_WORDS || h->layout != ISING_LAYOUT_COLUMN_INTERLEAVED ||
        !ci_valid_strips(h->g.L, nstrips))
        return ISING_EINVAL;
    h->chain = chain;
    h->nstrips = nstrips;
    return ISING_OK;
}

extern "C" int ising_sweep(ising_lattice* h, int64_t n)
{
    TraceRange trace("ising_sweep");
    if (!h || n < 0) return ISING_EINVAL;
    if (h->chain == ISING_CHAIN_RANDOM_WORDS) {
        while (n > 0) {
            const int64_t c = n > (1 << 30) ? (1 << 30) : n;
            int rc = run_random_words(h, c, [](int64_t) { return -1; });
            if (rc != ISING_OK) return rc;
            n -= c;
        }
        return ISING_OK;
    }
    if (use_resident(h)) {
        while (n > 0) {
            const int c = (int)std::min<int64_t>(n, 1 << 30);
            int rc = run_resident(h, c, 0x7fffffff);
            if (rc != ISING_OK) return rc;
            n -= c;
        }
        return ISING_OK;
    }
    ClusterPlan cp;
    if (use_cluster(h, &cp)) {
        while (n > 0) {
            const int64_t c = n > (1 << 30) ? (1 << 30) : n;
            int rc = run_cluster(h, c, 0, h->counts, cp);
            if (rc != ISING_OK) return rc;
            n -= c;
        }
        return ISING_OK;
    }
    if (use_graphs(h)) {
        int rc = replay_plain(h, &n);
        if (rc != ISING_OK) return rc;
    }
    // chunks keep t_off within 32 bits
    while (n > 0) {
        const int64_t c = n > (1 << 30) ? (1 << 30) : n;
        int rc = run_sweeps(h, c, [](int64_t) { return -1; });
        if (rc != ISING_OK) return rc;
        n -= c;
    }
    return ISING_OK;
}

static void counts_to_EM(const ising_lattice* h, const unsigned long long* slots, int64_t* E, int64_t* M)
{
    unsigned long long anti = 0, up = 0;
    for (int k = 0; k < kCountSlots; ++k) {
        anti += slots[2 * k];
        up += slots[2 * k + 1];
    }
    const int64_t N = (int64_t)h->g.L * h->g.L;
    if (E) *E = 2 * (int64_t)anti - 2 * N;
    if (M) *M = 2 * (int64_t)up - N;
}

extern "C" int ising_sweep_record(ising_lattice* h, int64_t n, int64_t every, int64_t* E, int64_t* M)
{
    TraceRange trace("ising_sweep_record");
    if (!h || n < 0 || every < 1 || every > (1 << 22)) return ISING_EINVAL;   // a chunk's offsets fit 32 bits
    const int64_t nrec = n / every;
    int64_t done_rec = 0;
    if (use_resident(h) && h->chain == ISING_CHAIN_CHECKERBOARD) {
        while (done_rec < nrec) {
            // at most 2^30 sweeps a launch
            const int64_t chunk = std::min<int64_t>({nrec - done_rec, (int64_t)kRecordsPerChunk, (1 << 30) / every});
            int rc = run_resident(h, (int)(chunk * every), (int)every);
            if (rc != ISING_OK) return rc;
            const size_t bytes = (size_t)chunk * 2 * sizeof(long long);
            cudaError_t e = cudaMemcpyAsync(h->host_counts, h->counts, bytes, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "resident records");
            const long long* rec = reinterpret_cast<const long long*>(h->host_counts);
            for (int64_t r = 0; r < chunk; ++r) {
                if (E) E[done_rec + r] = rec[2 * r];
                if (M) M[done_rec + r] = rec[2 * r + 1];
            }
            done_rec += chunk;
        }
        const int64_t rest = n - nrec * every;
        if (rest > 0) return ising_sweep(h, rest);
        return ISING_OK;
    }
    ClusterPlan cp;
    while (done_rec < nrec) {
        const int64_t chunk = (nrec - done_rec) < kRecordsPerChunk ? (nrec - done_rec) : kRecordsPerChunk;
        const size_t bytes = (size_t)chunk * kCountSlots * 2 * sizeof(unsigned long long);
        cudaError_t e = cudaMemsetAsync(h->counts, 0, bytes, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counts");
        int rc;
        if (h->chain == ISING_CHAIN_RANDOM_WORDS)
            rc = run_random_words(h, chunk * every, [every](int64_t s) {
                return (s % every == 0) ? (int)(s / every - 1) : -1;
            });
        else if (use_cluster(h, &cp))
            rc = run_cluster(h, chunk * every, every, h->counts, cp);
        else if (use_graphs(h) && every <= kGraphMaxEvery)
            rc = replay_records(h, chunk, (int)every);
        else
            rc = run_sweeps(h, chunk * every, [every](int64_t s) {
                return (s % every == 0) ? (int)(s / every - 1) : -1;
            });
        if (rc != ISING_OK) return rc;
        e = cudaMemcpyAsync(h->host_counts, h->counts, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync counts");
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        for (int64_t r = 0; r < chunk; ++r)
            counts_to_EM(h, h->host_counts + (size_t)r * kCountSlots * 2, E ? E + done_rec + r : nullptr,
                         M ? M + done_rec + r : nullptr);
        done_rec += chunk;
    }
    const int64_t rest = n - nrec * every;
    if (rest > 0) return ising_sweep(h, rest);
    return ISING_OK;
}

static int measure(ising_lattice* h, int64_t* E, int64_t* M)
{
    const size_t bytes = (size_t)kCountSlots * 2 * sizeof(unsigned long long);
    cudaError_t e = cudaMemsetAsync(h->counts, 0, bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync counts");
    SweepArgs a = base_args(h);
    a.counts = h->counts;
    e = launch_hs(h, 1, false, true, a);
    if (e != cudaSuccess) return cuda_fail(e, "measure");
    e = cudaMemcpyAsync(h->host_counts, h->counts, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync counts");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    counts_to_EM(h, h->host_counts, E, M);
    return ISING_OK;
}

extern "C" int ising_energy(ising_lattice* h, int64_t* E)
{
    if (!h || !E) return ISING_EINVAL;
    return measure(h, E, nullptr);
}

extern "C" int ising_magnetization(ising_lattice* h, int64_t* M)
{
    if (!h || !M) return ISING_EINVAL;
    return measure(h, nullptr, M);
}

// Eq. 2: exact 128-bit sums of the records, then one IEEE double division
// each (the integer count n L^2 converted once).
extern "C" int ising_means(const int64_t* E, const int64_t* M, int64_t n, int32_t L, double* mean_e,
                           double* mean_absm)
{
    if (n < 1 || !valid_L(L) || (!mean_e && !mean_absm) || (mean_e && !E) || (mean_absm && !M))
        return ISING_EINVAL;
    const double count = (double)((__int128)n * L * L);
    if (mean_e) {
        __int128 sum = 0;
        for (int64_t k = 0; k < n; ++k) sum += E[k];
        *mean_e = (double)sum / count;
    }
    if (mean_absm) {
        __int128 sum = 0;
        for (int64_t k = 0; k < n; ++k) sum += M[k] < 0 ? -(__int128)M[k] : (__int128)M[k];
        *mean_absm = (double)sum / count;
    }
    return ISING_OK;
}

static int ensure_staging(ising_lattice* h)
{
    if (h->staging) return ISING_OK;
    cudaError_t e = cudaMalloc(&h->staging, (size_t)h->g.L * h->g.L);
    if (e != cudaSuccess) { h->staging = nullptr; cuda_fail(e, "cudaMalloc staging"); return ISING_ENOMEM; }
    return ISING_OK;
}

extern "C" int ising_get_spins(ising_lattice* h, int8_t* out, size_t n)
{
    TraceRange trace("ising_get_spins");
    if (!h || !out || n != (size_t)h->g.L * h->g.L) return ISING_EINVAL;
    int rc = ensure_staging(h);
    if (rc != ISING_OK) return rc;
    const Geom& g = h->g;
    cudaError_t e;
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED) {
        e = ci_unpack(h->words[0], g.L, h->staging, h->stream);
    } else {
        e = launch_unpack(h->words[0], h->words[1], g, h->staging, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "unpack_kernel");
    e = cudaMemcpyAsync(out, h->staging, n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync spins");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return ISING_OK;
}

extern "C" int ising_set_spins(ising_lattice* h, const int8_t* in, size_t n)
{
    TraceRange trace("ising_set_spins");
    if (!h || !in || n != (size_t)h->g.L * h->g.L) return ISING_EINVAL;
    int rc = ensure_staging(h);
    if (rc != ISING_OK) return rc;
    const Geom& g = h->g;
    // Pinned host memory is read by the pack kernel itself (one pass over the
    // host link); anything else is first copied to the device staging buffer.
    const int8_t* src = h->staging;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, in);
    if (e == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer &&
        h->layout == ISING_LAYOUT_ROW_PACKED) {
        src = static_cast<const int8_t*>(attr.devicePointer);
    } else {
        cudaGetLastError();                          // a failed query is not an error here
        e = cudaMemcpyAsync(h->staging, in, n, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync spins");
    }
    if (h->layout == ISING_LAYOUT_COLUMN_INTERLEAVED) {
        e = ci_pack(h->words[0], g.L, h->staging, h->stream);
    } else {
        e = launch_pack_rows(h->words[0], h->words[1], g, src, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pack_rows_kernel");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return ISING_OK;
}

// Resources of ising_run_states (created on first use, kept): the second
// input buffer, a copy stream and the events that order copies, packs and
// sweeps.
static int ensure_pipeline(ising_lattice* h)
{
    int rc = ensure_staging(h);
    if (rc != ISING_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (!h->staging2) {
        e = cudaMalloc(&h->staging2, (size_t)h->g.L * h->g.L);
        if (e != cudaSuccess) { h->staging2 = nullptr; cuda_fail(e, "cudaMalloc staging"); return ISING_ENOMEM; }
    }
    if (!h->copy_stream) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if (!h->ev_copied[b]) e = cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_packed[b]) e = cudaEventCreateWithFlags(&h->ev_packed[b], cudaEventDisableTiming);
    }
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "run_states setup");
}

extern "C" int ising_run_states(ising_lattice* h, const int8_t* const* states, int32_t nstates, int64_t sweeps,
                                int64_t every, int64_t* E, int64_t* M)
{
    TraceRange trace("ising_run_states");
    if (!h || !states || nstates < 0 || sweeps < 0 || sweeps > (1 << 30) || every < 1 || every > (1 << 22))
        return ISING_EINVAL;
    for (int32_t k = 0; k < nstates; ++k)
        if (!states[k]) return ISING_EINVAL;
    const size_t nn = (size_t)h->g.L * h->g.L;
    const int64_t R = sweeps / every;                          // records per state
    if (h->layout != ISING_LAYOUT_ROW_PACKED || use_resident(h) || R > kRecordsPerChunk ||
        h->chain != ISING_CHAIN_CHECKERBOARD) {
        // no overlap to gain (on-chip path) or records beyond one chunk: the same calls in turn
        for (int32_t k = 0; k < nstates; ++k) {
            int rc = ising_set_spins(h, states[k], nn);
            if (rc == ISING_OK) rc = ising_sweep_record(h, sweeps, every, E ? E + k * R : nullptr, M ? M + k * R : nullptr);
            if (rc != ISING_OK) return rc;
        }
        return ISING_OK;
    }
    int rc = ensure_pipeline(h);
    if (rc != ISING_OK) return rc;
    const Geom& g = h->g;
    int8_t* stage[2] = {h->staging, h->staging2};
    const size_t rec_words = (size_t)kCountSlots * 2;         // count slots of one record
    const int64_t group = R > 0 ? std::max<int64_t>(1, kRecordsPerChunk / R) : (int64_t)nstates;
    for (int64_t k0 = 0; k0 < nstates; k0 += group) {
        const int64_t k1 = std::min<int64_t>(nstates, k0 + group);
        cudaError_t e = cudaSuccess;
        if (R > 0)
            e = cudaMemsetAsync(h->counts, 0, (size_t)(k1 - k0) * R * rec_words * sizeof(unsigned long long),
                                h->stream);
        for (int64_t k = k0; k < k1 && e == cudaSuccess; ++k) {
            const int b = (int)(k & 1);
            // state k -> input buffer b, once the pack that last read buffer b is done;
            // this copy runs while the sweeps of state k - 1 are on the device
            e = cudaStreamWaitEvent(h->copy_stream, h->ev_packed[b], 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(stage[b], states[k], nn, cudaMemcpyHostToDevice, h->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[b], h->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0);
            if (e != cudaSuccess) break;
            e = launch_pack_rows(h->words[0], h->words[1], g, stage[b], h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_packed[b], h->stream);
            if (e != cudaSuccess) break;
            const int64_t base = (k - k0) * R;
            ClusterPlan cp;
            if (use_cluster(h, &cp))
                rc = run_cluster(h, sweeps, every, h->counts + (size_t)base * rec_words, cp);
            else
                rc = run_sweeps(h, sweeps, [every, base](int64_t s) {
                    return (s % every == 0) ? (int)(base + s / every - 1) : -1;
                });
            if (rc != ISING_OK) return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "run_states");
        if (R > 0) {
            const size_t nrec = (size_t)(k1 - k0) * R;
            e = cudaMemcpyAsync(h->host_counts, h->counts, nrec * rec_words * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync counts");
        }
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        for (int64_t r = 0; r < (k1 - k0) * R; ++r)
            counts_to_EM(h, h->host_counts + (size_t)r * rec_words, E ? E + k0 * R + r : nullptr,
                         M ? M + k0 * R + r : nullptr);
    }
    return ISING_OK;
}

extern "C" int ising_get_words(ising_lattice* h, uint64_t* out, size_t n64)
{
    if (!h || !out) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    const size_t per = (size_t)h->g.L * h->g.P;
    if (n64 != 2 * per) return ISING_EINVAL;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpyAsync(out + c * per, h->words[c], per * sizeof(uint64_t),
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync words");
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "cudaStreamSynchronize");
}

extern "C" int ising_set_words(ising_lattice* h, const uint64_t* in, size_t n64)
{
    if (!h || !in) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    const size_t per = (size_t)h->g.L * h->g.P;
    if (n64 != 2 * per) return ISING_EINVAL;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpyAsync(h->words[c], in + c * per, per * sizeof(uint64_t),
                                        cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync words");
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "cudaStreamSynchronize");
}

extern "C" int ising_layout(ising_lattice* h, int32_t* W, int32_t* pitch, int32_t* last_fields)
{
    if (!h) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    if (W) *W = h->g.W;
    if (pitch) *pitch = h->g.P;
    if (last_fields) *last_fields = h->g.rlast;
    return ISING_OK;
}

extern "C" int ising_get_sweep(ising_lattice* h, uint64_t* t)
{
    if (!h || !t) return ISING_EINVAL;
    *t = h->t;
    return ISING_OK;
}

extern "C" int ising_set_sweep(ising_lattice* h, uint64_t t)
{
    if (!h) return ISING_EINVAL;
    return reset_t(h, t);
}

extern "C" int ising_set_stream(ising_lattice* h, void* stream)
{
    if (!h) return ISING_EINVAL;
    h->stream = (cudaStream_t)stream;
    return ISING_OK;
}

extern "C" int ising_set_tiling(ising_lattice* h, int32_t rows, int32_t bw, int32_t bgrp)
{
    if (!h) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    if (rows != 4) return ISING_EINVAL;
    if (bw == 0) {                                  // linear items, bgrp threads per block
        if (bgrp != 64 && bgrp != 128 && bgrp != 192 && bgrp != 256) return ISING_EINVAL;
        h->bw = 0;
        h->bg = bgrp;
        drop_graphs(h);
        return ISING_OK;
    }
    if (bw != 16 && bw != 32 && bw != 64) return ISING_EINVAL;
    if (bgrp != 1 && bgrp != 2 && bgrp != 4 && bgrp != 8 && bgrp != 16) return ISING_EINVAL;
    if (bw * bgrp > 256 || bw * bgrp < 32) return ISING_EINVAL;
    h->bw = bw;
    h->bg = bgrp;
    drop_graphs(h);
    return ISING_OK;
}

extern "C" int ising_set_item_lanes(ising_lattice* h, int32_t lanes)
{
    if (!h) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return ISING_EINVAL;
    h->item_lanes = lanes;
    drop_graphs(h);
    return ISING_OK;
}

extern "C" int ising_device_words(ising_lattice* h, int32_t c, void** dev_ptr)
{
    if (!h || !dev_ptr || (c != 0 && c != 1)) return ISING_EINVAL;
    if (h->layout != ISING_LAYOUT_ROW_PACKED) return ISING_EINVAL;   // row-packed words only
    *dev_ptr = h->words[c];
    return ISING_OK;
}

extern "C" int ising_philox_blocks(uint64_t seed, const uint32_t* host_ctr, uint32_t* host_out, int64_t n)
{
    if (!host_ctr || !host_out || n < 0 || n > (1 << 24)) return ISING_EINVAL;
    if (n == 0) return ISING_OK;
    uint32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)n * 8 * sizeof(uint32_t));
    if (e != cudaSuccess) { cuda_fail(e, "cudaMalloc"); return ISING_ENOMEM; }
    int rc = ISING_OK;
    e = cudaMemcpy(d, host_ctr, (size_t)n * 4 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        e = launch_philox_blocks(d, d + 4 * n, n, seed, nullptr);
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d + 4 * n, (size_t)n * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "philox_blocks");
    cudaFree(d);
    return rc;
}

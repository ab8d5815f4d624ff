// Device kernels of the single-lattice path and their launchers: hot/cold
// initialisation, spin packing, the half-sweep kernels of the launch path
// (one thread per item, or F lanes per item), the on-chip kernels, the sweep
// counter kernels and the Philox test hook; plus the host helpers shared by
// the library (thresholds, launch arguments, geometry, error recording).
// The C ABI that drives them: ising_lattice.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <type_traits>

#include "../../include/ising.h"
#include "ising_device.cuh"
#include "ising_internal.h"

namespace ising {

// The checked build's readers of each translation unit's out-of-range word
// (see check_index in ising_device.cuh); a function-local table, so that the
// registrations made while the library loads need no initialisation order.
namespace {
constexpr int kMaxCheckReaders = 16;
struct CheckReaders {
    int (*fn[kMaxCheckReaders])(unsigned long long*) = {};
    int n = 0;
};
CheckReaders& check_readers()
{
    static CheckReaders r;
    return r;
}
}  // namespace

bool register_check_reader(int (*reader)(unsigned long long*))
{
    CheckReaders& r = check_readers();
    if (r.n < kMaxCheckReaders) r.fn[r.n++] = reader;
    return true;
}

// Hot start: s = +1 iff the site's Philox draw at t = 0 is below 2^31.
// Thread = (4-row group, word, colour).
__global__ void init_hot_kernel(uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, Geom g,
                                uint32_t key0, uint32_t key1)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y * blockDim.y + threadIdx.y;
    const int c = blockIdx.z;
    if (w >= g.W || grp * 4 >= g.L) return;
    const uint64_t live = live_mask(g, w);
    uint64_t word[4] = {0, 0, 0, 0};
    for (int k = 0; k < kFields; ++k) {
        uint32_t x[4] = {(uint32_t)grp, (uint32_t)(w * kFields + k), 0u, (uint32_t)c};
        philox10(x, key0, key1);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            word[e] |= (uint64_t)((x[e] >> 31) ^ 1u) << (3 * k);
    }
    uint64_t* arr = c ? w1 : w0;
    for (int e = 0; e < 4; ++e) {
        const int i = grp * 4 + e;
        if (i < g.L) arr[(size_t)i * g.P + w] = word[e] & live;
    }
}

// Cold start (all up or all down); also zeroes the pitch padding.
__global__ void init_cold_kernel(uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, Geom g, int up)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (w >= g.P || i >= g.L) return;
    const uint64_t v = (w < g.W && up) ? live_mask(g, w) : 0ull;
    w0[(size_t)i * g.P + w] = v;
    w1[(size_t)i * g.P + w] = v;
}

// int8 spins of row blockIdx.x (> 0 is up) -> that row's words of both
// colours.  The row is first staged in shared memory (16-byte loads when
// vec16: `in` 16-byte aligned and L % 16 == 0), so the input is read once
// and coalesced; `in` may be device memory or pinned host memory mapped into
// the device's address space.  Dynamic shared memory: L bytes.
__global__ void pack_rows_kernel(uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, Geom g,
                                 const int8_t* __restrict__ in, int vec16)
{
    extern __shared__ __align__(16) int8_t row_s[];
    const int i = blockIdx.x;
    const int8_t* src = in + (size_t)i * g.L;
    if (vec16) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(row_s);
        for (int k = threadIdx.x; k < g.L / 16; k += blockDim.x) d4[k] = s4[k];
    } else {
        for (int k = threadIdx.x; k < g.L; k += blockDim.x) row_s[k] = src[k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * g.P; t += blockDim.x) {
        const int c = t >= g.P ? 1 : 0;
        const int w = t - c * g.P;
        uint64_t word = 0;
        if (w < g.W) {
            const int nf = (w == g.W - 1) ? g.rlast : kFields;
            const int par = (i + c) & 1;
            const int8_t* r = row_s + 2 * w * kFields + par;
            for (int k = 0; k < nf; ++k) word |= (uint64_t)(r[2 * k] > 0) << (3 * k);
        }
        (c ? w1 : w0)[(size_t)i * g.P + w] = word;
    }
}

// Packed colour words -> int8 spins (+1 / -1).
__global__ void unpack_kernel(const uint64_t* __restrict__ w0, const uint64_t* __restrict__ w1, Geom g,
                              int8_t* __restrict__ s)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int c = blockIdx.z;
    if (w >= g.W || i >= g.L) return;
    const uint64_t word = (c ? w1 : w0)[(size_t)i * g.P + w];
    const int nf = (w == g.W - 1) ? g.rlast : kFields;
    const int par = (i + c) & 1;
    int8_t* row = s + (size_t)i * g.L;
    for (int k = 0; k < nf; ++k) {
        const int j = 2 * (w * kFields + k) + par;
        row[j] = ((word >> (3 * k)) & 1ull) ? (int8_t)1 : (int8_t)-1;
    }
}

// t_base += n (end of a chunk of sweeps).
__global__ void advance_sweep_kernel(uint64_t* t_base, uint64_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t_base += n;
}

// End of a replayed graph of sweeps: t_base += n, record index += inc.
__global__ void advance_graph_kernel(uint64_t* t_base, uint64_t n, uint32_t* rec_base, uint32_t inc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *t_base += n;
        *rec_base += inc;
    }
}

__global__ void set_sweep_kernel(uint64_t* t_base, uint64_t t)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t_base = t;
}

// Temporal blocking with the whole lattice on chip: one block copies both
// colour arrays into shared memory, runs sweeps t0+1 .. t0+n there (a block
// barrier between half-sweeps), records E and M after every `every`-th sweep
// with an on-chip reduction (records[2k] = E, records[2k+1] = M), and copies
// the lattice back.  For lattices whose 2 L P words fit in shared memory.
template <int ROUNDS>
__global__ void __launch_bounds__(256, 1)
resident_sweeps_kernel(uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, Geom g, SweepArgs a, uint64_t t0,
                       int n, int every, long long* __restrict__ records)
{
    extern __shared__ __align__(16) uint64_t lattice[];
    __shared__ unsigned int red_anti[8], red_up[8];
    const size_t words = (size_t)g.L * g.P;
    uint64_t* s0 = lattice;
    uint64_t* s1 = lattice + words;
    for (size_t k = threadIdx.x; k < words; k += blockDim.x) {
        s0[k] = w0[k];
        s1[k] = w1[k];
    }
    __syncthreads();
    const int items = ((g.L + 3) / 4) * g.W;
    const long long N = (long long)g.L * g.L;
    for (int s = 1; s <= n; ++s) {
        const uint64_t t = t0 + (uint64_t)s;
        uint32_t dummy0 = 0, dummy1 = 0;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int grp = it / g.W, w = it - grp * g.W;
            sweep_rows<0, true, false, false, ROUNDS>(s0, s1, g, grp * 4, w, t, a.rk, a.thr0, a.thr1, a.all0,
                                                      a.all1, a.one, dummy0, dummy1);
        }
        __syncthreads();
        const bool record = (s % every) == 0;
        uint32_t anti = 0, up = 0;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int grp = it / g.W, w = it - grp * g.W;
            if (record)
                sweep_rows<1, true, true, false, ROUNDS>(s1, s0, g, grp * 4, w, t, a.rk, a.thr0, a.thr1, a.all0,
                                                         a.all1, a.one, anti, up);
            else
                sweep_rows<1, true, false, false, ROUNDS>(s1, s0, g, grp * 4, w, t, a.rk, a.thr0, a.thr1, a.all0,
                                                          a.all1, a.one, anti, up);
        }
        if (record) {
            anti = __reduce_add_sync(0xffffffffu, anti);
            up = __reduce_add_sync(0xffffffffu, up);
            if ((threadIdx.x & 31) == 0) { red_anti[threadIdx.x >> 5] = anti; red_up[threadIdx.x >> 5] = up; }
        }
        __syncthreads();
        if (record && threadIdx.x == 0) {
            unsigned long long sa = 0, su = 0;
            for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) { sa += red_anti[k]; su += red_up[k]; }
            const int rec = s / every - 1;
            records[2 * rec] = 2 * (long long)sa - 2 * N;
            records[2 * rec + 1] = 2 * (long long)su - N;
        }
    }
    __syncthreads();
    for (size_t k = threadIdx.x; k < words; k += blockDim.x) {
        w0[k] = s0[k];
        w1[k] = s1[k];
    }
}

// Accept masks of the sweeps j = 0 .. nsweeps-1 that follow sweep t0 (sweep
// t0 + j + 1), one thread per (j, item), drawn exactly as sweep_rows draws
// them: masks[(j * items + item) * 4 + e] = (colour-0, colour-1 packed masks)
// of row e of the item (item_masks_thread).  The draws depend on the site,
// sweep and colour only, so a whole run's masks can be drawn at once by every
// SM before the spins are updated.  t_base (device memory, or null) is added
// to t0: a graph that is replayed draws for the sweeps after the device sweep
// counter.
template <int ROUNDS>
__global__ void __launch_bounds__(128)
mask_draw_kernel(Geom g, SweepArgs a, const uint64_t* t_base, uint64_t t0, int nsweeps, ulonglong2* __restrict__ masks)
{
    const int items = ((g.L + 3) / 4) * g.W;
    const long long total = (long long)nsweeps * items;
    const uint64_t tb = (t_base ? *t_base : 0) + t0 + 1;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / items);
        const int item = (int)(k - (long long)j * items);
        uint64_t p0[4], p1[4];
        const uint64_t t = tb + (uint64_t)j;
        item_masks_thread<ROUNDS>(g, item, t, 0, a.rk, a.thr0, a.thr1, a.one, p0);
        item_masks_thread<ROUNDS>(g, item, t, 1, a.rk, a.thr0, a.thr1, a.one, p1);
        ulonglong2* out = masks + (size_t)k * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) out[e] = make_ulonglong2(p0[e], p1[e]);
    }
}

// The on-chip path with the masks drawn beforehand (mask_draw_kernel): one
// block holds the lattice in shared memory and runs sweeps s_base+1 ..
// s_base+n of a run.  Thread x updates the rows (item, e) numbered 4 item + e
// = x, x + blockDim.x, ... (R of them) in every half-sweep.  Their masks (one
// 16-byte load per row and sweep) are read from global memory two sweeps
// ahead, so a half-sweep's critical path is the spin logic of R rows and one
// barrier; the Philox work ran beforehand on all SMs.  Each warp adds its
// E/M counts of a recorded sweep to shared memory with one atomic per count;
// the records of the run (after its sweeps s with s % every == 0) are
// written at the end to records[2 (s / every - 1) ..] as (E, M).  rec_first
// is the first record of this launch and nrec their number; the dynamic
// shared memory holds both colour arrays and 2 nrec counters.  Same results
// as resident_sweeps_kernel.  H = 2 splits every row over two threads, one
// per 32-bit half of its word (row_half_apply): twice the warps for a small
// lattice, each with half of the spin logic.
template <int R, int H>
__global__ void __launch_bounds__(1024, 1)
resident_premasked_kernel(uint64_t* __restrict__ w0, uint64_t* __restrict__ w1, Geom g, SweepArgs a, int s_base,
                          int n, int every, int rec_first, int nrec, const ulonglong2* __restrict__ masks,
                          long long* __restrict__ records)
{
    extern __shared__ __align__(16) uint64_t lattice[];
    const size_t words = (size_t)g.L * g.P;
    uint64_t* s0 = lattice;
    uint64_t* s1 = lattice + words;
    unsigned int* rec_sm = reinterpret_cast<unsigned int*>(lattice + 2 * words);
    for (size_t k = threadIdx.x; k < words; k += blockDim.x) {
        s0[k] = w0[k];
        s1[k] = w1[k];
    }
    for (int k = threadIdx.x; k < 2 * nrec; k += blockDim.x) rec_sm[k] = 0;
    __syncthreads();
    const int items = ((g.L + 3) / 4) * g.W;
    const size_t stride = (size_t)items * 4;             // masks of one sweep
    const ulonglong2 zero = make_ulonglong2(0, 0);
    int row[R], col[R];
    bool valid[R];
    uint64_t live[R], all0[R], all1[R];
    // packed masks (colour 0, colour 1) of sweep s (c) and s + 1 (nx) of each row
    ulonglong2 c[R], nx[R];
    int mi[R], hf[R];                    // the unit's mask entry (its row) and word half (H = 2)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int x = (int)threadIdx.x + r * (int)blockDim.x;
        mi[r] = x / H;
        hf[r] = x % H;
        const int item = mi[r] >> 2, e = mi[r] & 3;
        const int grp = item / g.W;
        col[r] = item - grp * g.W;
        row[r] = grp * 4 + e;
        valid[r] = item < items && row[r] < g.L;
        live[r] = valid[r] ? live_mask(g, col[r]) : 0;
        all0[r] = ((uint64_t)a.all0 << 32 | a.all0) & live[r];
        all1[r] = ((uint64_t)a.all1 << 32 | a.all1) & live[r];
        c[r] = nx[r] = zero;
        if (valid[r]) {
            c[r] = __ldg(masks + mi[r]);
            if (n >= 2) nx[r] = __ldg(masks + stride + mi[r]);
        }
    }
    // one half-sweep of unit r with the packed masks p of its row
    auto apply = [&](auto colour, auto rec, int r, uint64_t p, uint32_t& anti, uint32_t& up) {
        constexpr int C = decltype(colour)::value;
        constexpr bool REC = decltype(rec)::value;
        if constexpr (H == 1) {
            row_apply<C, REC>(C == 0 ? s0 : s1, C == 0 ? s1 : s0, g, row[r], col[r], live[r], p, p >> 1, all0[r],
                              all1[r], anti, up);
        } else {
            const int sh = 32 * hf[r];
            row_half_apply<C, REC>(C == 0 ? s0 : s1, C == 0 ? s1 : s0, g, row[r], col[r], hf[r],
                                   (uint32_t)(live[r] >> sh), (uint32_t)(p >> sh), (uint32_t)((p >> 1) >> sh),
                                   (uint32_t)(all0[r] >> sh), (uint32_t)(all1[r] >> sh), anti, up);
        }
    };
    // the next recorded sweep of this launch and its slot in rec_sm
    int next = every - s_base % every;
    int slot = 0;
    for (int s = 1; s <= n; ++s) {
        ulonglong2 f[R];
        uint32_t anti = 0, up = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            f[r] = zero;
            if (valid[r] && s + 2 <= n) f[r] = __ldg(masks + (size_t)(s + 1) * stride + mi[r]);
            if (valid[r]) apply(std::integral_constant<int, 0>(), std::false_type(), r, c[r].x, anti, up);
        }
        __syncthreads();
        const bool record = s == next;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (valid[r]) {
                if (record) apply(std::integral_constant<int, 1>(), std::true_type(), r, c[r].y, anti, up);
                else apply(std::integral_constant<int, 1>(), std::false_type(), r, c[r].y, anti, up);
            }
            c[r] = nx[r];
            nx[r] = f[r];
        }
        if (record) {
            anti = __reduce_add_sync(0xffffffffu, anti);
            up = __reduce_add_sync(0xffffffffu, up);
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(rec_sm + 2 * slot, anti);
                atomicAdd(rec_sm + 2 * slot + 1, up);
            }
            next += every;
            ++slot;
        }
        __syncthreads();
    }
    const long long N = (long long)g.L * g.L;
    for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
        records[2 * (rec_first + k)] = 2 * (long long)rec_sm[2 * k] - 2 * N;
        records[2 * (rec_first + k) + 1] = 2 * (long long)rec_sm[2 * k + 1] - N;
    }
    for (size_t k = threadIdx.x; k < words; k += blockDim.x) {
        w0[k] = s0[k];
        w1[k] = s1[k];
    }
}

// One half-sweep of colour C over all SMs with the masks drawn beforehand
// (mask_draw_kernel): thread k updates row k & 3 of item k >> 2 with the
// packed masks masks[k] (.x colour 0, .y colour 1), so a launch is short:
// no Philox work, one row of spin logic per thread.  Same results as
// half_sweep_kernel.
template <int C, bool RECORD>
__global__ void __launch_bounds__(128)
half_sweep_apply_kernel(uint64_t* __restrict__ own, const uint64_t* __restrict__ other, Geom g, SweepArgs a,
                        const ulonglong2* __restrict__ masks)
{
    pdl_enter();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int items = ((g.L + 3) / 4) * g.W;
    const int item = (int)(k >> 2), e = (int)(k & 3);
    const int grp = item / g.W;
    const int w = item - grp * g.W;
    const int i = grp * 4 + e;
    uint32_t anti = 0, up = 0;
    if (item < items && i < g.L) {
        const uint64_t live = live_mask(g, w);
        const uint64_t all0 = ((uint64_t)a.all0 << 32 | a.all0) & live;
        const uint64_t all1 = ((uint64_t)a.all1 << 32 | a.all1) & live;
        const uint64_t p = C == 0 ? __ldg(&masks[k].x) : __ldg(&masks[k].y);
        row_apply<C, RECORD>(own, other, g, i, w, live, p, p >> 1, all0, all1, anti, up);
    }
    if (RECORD) block_add_counts(record_counts(a) + 2 * (blockIdx.x % kCountSlots), anti, up);
}

cudaError_t launch_half_sweep_apply(int colour, bool record, uint64_t* own, const uint64_t* other, const Geom& g,
                                    const SweepArgs& a, const ulonglong2* masks, cudaStream_t s)
{
    const uint32_t threads = (uint32_t)(((g.L + 3) / 4) * g.W) * 4;
    const dim3 block(128), grid((threads + 127) / 128);
    // Programmatic dependent launch also inside the captured graphs, where the
    // fused half-sweeps use plain launches: measured on GB300 against plain
    // launches in the same graphs (sweeps without records, spin-updates/ns),
    // L = 300 / 512 / 700 / 1008: 35 / 97 / 171 / 314 against 31 / 87 / 156 /
    // 294, and L = 4096: 1006 against 963, but L = 1500 / 2016 / 2600: 499 /
    // 651 / 782 against 508 / 681 / 816 (L = 3000: equal).  So it is on up to
    // 8192 items and from 80000 items.
    const int items = ((g.L + 3) / 4) * g.W;
    const bool in_graphs = items <= 8192 || items >= 80000;
    if (colour == 0)
        launch_pdl_opt(in_graphs, half_sweep_apply_kernel<0, false>, grid, block, s, own, other, g, a, masks);
    else if (record)
        launch_pdl_opt(in_graphs, half_sweep_apply_kernel<1, true>, grid, block, s, own, other, g, a, masks);
    else
        launch_pdl_opt(in_graphs, half_sweep_apply_kernel<1, false>, grid, block, s, own, other, g, a, masks);
    return cudaGetLastError();
}

// One half-sweep of colour C over all SMs with F lanes per thread item
// (sweep_item_lanes on the lattice in global memory): for lattices whose one
// thread per item would leave SMs idle and each thread with a long chain of
// 21 Philox calls.  Thread k of the grid is lane k % F of item k / F.  Same
// results as half_sweep_kernel.
template <int C, bool RECORD, int F, int ROUNDS>
__global__ void __launch_bounds__(128, 4)
half_sweep_lanes_kernel(uint64_t* __restrict__ own, const uint64_t* __restrict__ other, Geom g, SweepArgs a)
{
    pdl_enter();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = (int)(k / F), q = (int)(k % F);
    const int items = ((g.L + 3) / 4) * g.W;
    const uint64_t t = *a.t_base + a.t_off;
    uint32_t anti = 0, up = 0;
    sweep_item_lanes<C, RECORD, F, ROUNDS>(own, other, g, item, item < items, q, t, a.rk, a.thr0, a.thr1, a.all0,
                                           a.all1, anti, up);
    if (RECORD) block_add_counts(record_counts(a) + 2 * (blockIdx.x % kCountSlots), anti, up);
}

template <int F, int ROUNDS>
static void launch_lanes_r(int colour, bool record, uint64_t* own, const uint64_t* other, const Geom& g,
                           const SweepArgs& a, cudaStream_t s)
{
    const uint32_t threads = (uint32_t)(((g.L + 3) / 4) * g.W) * F;
    const dim3 block(128), grid((threads + 127) / 128);
    if (colour == 0) launch_pdl(half_sweep_lanes_kernel<0, false, F, ROUNDS>, grid, block, s, own, other, g, a);
    else if (record) launch_pdl(half_sweep_lanes_kernel<1, true, F, ROUNDS>, grid, block, s, own, other, g, a);
    else launch_pdl(half_sweep_lanes_kernel<1, false, F, ROUNDS>, grid, block, s, own, other, g, a);
}

// A half-sweep that updates, with F = 2, 4 or 8 lanes per item.
cudaError_t launch_half_sweep_lanes(int F, int colour, bool record, uint64_t* own, const uint64_t* other,
                                    const Geom& g, const SweepArgs& a, cudaStream_t s)
{
    const bool r7 = a.rounds == 7;
    switch (F) {
    case 2: r7 ? launch_lanes_r<2, 7>(colour, record, own, other, g, a, s)
               : launch_lanes_r<2, 10>(colour, record, own, other, g, a, s); break;
    case 4: r7 ? launch_lanes_r<4, 7>(colour, record, own, other, g, a, s)
               : launch_lanes_r<4, 10>(colour, record, own, other, g, a, s); break;
    default: r7 ? launch_lanes_r<8, 7>(colour, record, own, other, g, a, s)
                : launch_lanes_r<8, 10>(colour, record, own, other, g, a, s); break;
    }
    return cudaGetLastError();
}

// Test hook: Philox4x32-10 blocks of arbitrary counters.
__global__ void philox_blocks_kernel(const uint32_t* __restrict__ ctr, uint32_t* __restrict__ out,
                                     int64_t n, uint32_t key0, uint32_t key1)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint32_t x[4] = {ctr[4 * b], ctr[4 * b + 1], ctr[4 * b + 2], ctr[4 * b + 3]};
    philox10(x, key0, key1);
    for (int e = 0; e < 4; ++e) out[4 * b + e] = x[e];
}

}  // namespace ising

namespace ising {

constexpr int kMaxSide = 32768;

thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char* where)
{
    snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", where, cudaGetErrorString(e));
    return ISING_ECUDA;
}

// Integer thresholds of Sec. 2 step 3 with dE = 8 - 4a (Table 1).
void thresholds_for_beta(double beta, uint64_t thr[2])
{
    const double two32 = 4294967296.0;
    for (int a = 0; a < 2; ++a) {
        const double dE = 8.0 - 4.0 * a;
        double x = std::floor(std::exp(-dE * beta) * two32);
        if (x > two32) x = two32;
        if (!(x >= 0.0)) x = 0.0;
        thr[a] = (uint64_t)x;
    }
}

void fill_threshold_args(const uint64_t thr[2], SweepArgs& a)
{
    const uint64_t two32 = 1ull << 32;
    a.thr0 = thr[0] >= two32 ? 0xFFFFFFFFu : (uint32_t)thr[0];
    a.thr1 = thr[1] >= two32 ? 0xFFFFFFFFu : (uint32_t)thr[1];
    a.all0 = thr[0] >= two32 ? 0xFFFFFFFFu : 0u;
    a.all1 = thr[1] >= two32 ? 0xFFFFFFFFu : 0u;
}

Geom lattice_geom(int L)
{
    Geom g;
    g.L = L;
    const int half = L / 2;
    g.W = (half + kFields - 1) / kFields;
    g.P = (g.W + 1) & ~1;
    g.rlast = half - kFields * (g.W - 1);
    return g;
}

bool valid_side(int32_t L) { return L >= 4 && L <= kMaxSide && (L % 2) == 0; }

cudaError_t launch_init_hot(uint64_t* w0, uint64_t* w1, const Geom& g, uint64_t seed, cudaStream_t s)
{
    dim3 block(32, 4);
    dim3 grid((g.W + 31) / 32, ((g.L + 3) / 4 + 3) / 4, 2);
    init_hot_kernel<<<grid, block, 0, s>>>(w0, w1, g, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_init_cold(uint64_t* w0, uint64_t* w1, const Geom& g, int up, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((g.P + 31) / 32, (g.L + 7) / 8);
    init_cold_kernel<<<grid, block, 0, s>>>(w0, w1, g, up);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint64_t* w0, const uint64_t* w1, const Geom& g, int8_t* out, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((g.W + 31) / 32, (g.L + 7) / 8, 2);
    unpack_kernel<<<grid, block, 0, s>>>(w0, w1, g, out);
    return cudaGetLastError();
}

SweepArgs make_sweep_args(uint64_t seed, const uint64_t thr[2], const uint64_t* t_base)
{
    SweepArgs a;
    a.t_base = t_base;
    a.t_off = 0;
    fill_threshold_args(thr, a);
    a.one = 1;
    a.rounds = 10;
    a.rk = philox_keys((uint32_t)seed, (uint32_t)(seed >> 32));
    a.counts = nullptr;
    a.rec_base = nullptr;
    return a;
}

template <int ROUNDS, bool LIN>
static void launch_half_sweep_r(dim3 grid, dim3 block, int colour, bool update, bool record, uint64_t* own,
                                const uint64_t* other, const Geom& g, const SweepArgs& a, cudaStream_t s)
{
    if (colour == 0) {
        if (record) launch_pdl(half_sweep_kernel<0, true, true, ROUNDS, LIN>, grid, block, s, own, other, g, a);
        else launch_pdl(half_sweep_kernel<0, true, false, ROUNDS, LIN>, grid, block, s, own, other, g, a);
    } else if (!update) {
        half_sweep_kernel<1, false, true, 10, LIN><<<grid, block, 0, s>>>(own, other, g, a);
    } else {
        if (record) launch_pdl(half_sweep_kernel<1, true, true, ROUNDS, LIN>, grid, block, s, own, other, g, a);
        else launch_pdl(half_sweep_kernel<1, true, false, ROUNDS, LIN>, grid, block, s, own, other, g, a);
    }
}

// bw == 0: linear items, bgrp threads per block; else bw x bgrp 2-D blocks.
cudaError_t launch_half_sweep(int bw, int bgrp, int colour, bool update, bool record,
                              uint64_t* own, const uint64_t* other, const Geom& g, const SweepArgs& a,
                              cudaStream_t s)
{
    const int ngroups = (g.L + 3) / 4;
    if (bw == 0) {
        const uint32_t items = (uint32_t)ngroups * (uint32_t)g.W;
        dim3 block(bgrp), grid((items + bgrp - 1) / bgrp);
        if (a.rounds == 7) launch_half_sweep_r<7, true>(grid, block, colour, update, record, own, other, g, a, s);
        else launch_half_sweep_r<10, true>(grid, block, colour, update, record, own, other, g, a, s);
        return cudaGetLastError();
    }
    dim3 block(bw, bgrp);
    dim3 grid((g.W + bw - 1) / bw, (ngroups + bgrp - 1) / bgrp);
    if (a.rounds == 7) launch_half_sweep_r<7, false>(grid, block, colour, update, record, own, other, g, a, s);
    else launch_half_sweep_r<10, false>(grid, block, colour, update, record, own, other, g, a, s);
    return cudaGetLastError();
}

}  // namespace ising

namespace ising {

cudaError_t launch_pack_rows(uint64_t* w0, uint64_t* w1, const Geom& g, const int8_t* src, cudaStream_t s)
{
    const int vec16 = ((uintptr_t)src % 16 == 0) && (g.L % 16 == 0);
    pack_rows_kernel<<<g.L, 256, g.L, s>>>(w0, w1, g, src, vec16);
    return cudaGetLastError();
}

cudaError_t launch_advance_sweep(uint64_t* t_base, uint64_t n, cudaStream_t s)
{
    advance_sweep_kernel<<<1, 1, 0, s>>>(t_base, n);
    return cudaGetLastError();
}

cudaError_t launch_advance_graph(uint64_t* t_base, uint64_t n, uint32_t* rec_base, uint32_t inc, cudaStream_t s)
{
    advance_graph_kernel<<<1, 1, 0, s>>>(t_base, n, rec_base, inc);
    return cudaGetLastError();
}

cudaError_t launch_set_sweep(uint64_t* t_base, uint64_t t, cudaStream_t s)
{
    set_sweep_kernel<<<1, 1, 0, s>>>(t_base, t);
    return cudaGetLastError();
}

cudaError_t launch_philox_blocks(const uint32_t* ctr, uint32_t* out, int64_t n, uint64_t seed, cudaStream_t s)
{
    philox_blocks_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, out, n, (uint32_t)seed,
                                                                    (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t allow_resident_smem(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(resident_sweeps_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resident_sweeps_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resident_premasked_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resident_premasked_kernel<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resident_premasked_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t launch_resident(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a, uint64_t t0, int n,
                            int every, long long* rec, size_t bytes, cudaStream_t s)
{
    const int items = ((g.L + 3) / 4) * g.W;
    const int threads = std::min(256, std::max(32, (items + 31) / 32 * 32));
    if (a.rounds == 7) resident_sweeps_kernel<7><<<1, threads, bytes, s>>>(w0, w1, g, a, t0, n, every, rec);
    else resident_sweeps_kernel<10><<<1, threads, bytes, s>>>(w0, w1, g, a, t0, n, every, rec);
    return cudaGetLastError();
}

int device_sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    return sms;
}

// Masks of the nsweeps sweeps following sweep (t_base ? *t_base : 0) + t0
// into `masks` (nsweeps * items * 4 entries), with at most
// blocks_per_sm * (the device's SMs) blocks of 128 threads (0: one thread
// per sweep and item).
cudaError_t launch_mask_draw(const Geom& g, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                             ulonglong2* masks, int blocks_per_sm, cudaStream_t s)
{
    const long long threads = (long long)nsweeps * (((g.L + 3) / 4) * g.W);
    unsigned blocks = (unsigned)((threads + 127) / 128);
    if (blocks_per_sm > 0) blocks = std::min(blocks, (unsigned)(device_sm_count() * blocks_per_sm));
    if (a.rounds == 7) mask_draw_kernel<7><<<blocks, 128, 0, s>>>(g, a, t_base, t0, nsweeps, masks);
    else mask_draw_kernel<10><<<blocks, 128, 0, s>>>(g, a, t_base, t0, nsweeps, masks);
    return cudaGetLastError();
}

cudaError_t launch_resident_premasked(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a, int s_base,
                                      int n, int every, const ulonglong2* masks, long long* rec, size_t bytes,
                                      cudaStream_t s)
{
    const int items = ((g.L + 3) / 4) * g.W;
    const int H = premasked_threads_per_row(items);
    const int R = premasked_rows_per_thread(items);
    const int threads = ((4 * H * items + R - 1) / R + 31) / 32 * 32;
    const int rec_first = s_base / every;
    const int nrec = (s_base + n) / every - rec_first;
    const size_t smem = bytes + 2 * (size_t)nrec * sizeof(unsigned int);
    if (H == 2)
        resident_premasked_kernel<1, 2><<<1, threads, smem, s>>>(w0, w1, g, a, s_base, n, every, rec_first, nrec,
                                                                 masks, rec);
    else if (R == 1)
        resident_premasked_kernel<1, 1><<<1, threads, smem, s>>>(w0, w1, g, a, s_base, n, every, rec_first, nrec,
                                                                 masks, rec);
    else
        resident_premasked_kernel<2, 1><<<1, threads, smem, s>>>(w0, w1, g, a, s_base, n, every, rec_first, nrec,
                                                                 masks, rec);
    return cudaGetLastError();
}

}  // namespace ising

extern "C" const char* ising_last_cuda_error(void) { return ising::g_last_cuda_error; }

extern "C" int ising_check_status(int32_t* checked, uint64_t* first_violation)
{
#ifdef ISING_CHECKED
    if (checked) *checked = 1;
#else
    if (checked) *checked = 0;
#endif
    if (first_violation) *first_violation = 0;
    ising::CheckReaders& r = ising::check_readers();
    if (r.n == 0) return ISING_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return ising::cuda_fail(e, "ising_check_status");
    for (int k = 0; k < r.n; ++k) {
        unsigned long long word = 0;
        if (r.fn[k](&word) != 0) return ising::cuda_fail(cudaGetLastError(), "ising_check_status");
        if (word && first_violation && *first_violation == 0) *first_violation = word;
    }
    return ISING_OK;
}

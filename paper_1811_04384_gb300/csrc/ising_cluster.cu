// Cluster-resident temporal blocking for mid-size lattices (above the
// one-SM on-chip range, L of about 130 to 3000).
//
// There a half-sweep is short: a replayed graph node per half-sweep costs
// more than its work.  Here one launch of G thread-block clusters (of 16
// blocks where the device allows it, else 8) runs a piece of up to 256
// sweeps whose accept masks cl_mask_draw_kernel draws on the SMs the
// clusters leave free.  The launch's G C blocks own consecutive row bands of
// both colours, block B rows B L / (G C) .. (B + 1) L / (G C) - 1, and keep
// them in shared memory for the whole launch, in a window with k rows of
// halo above and below (k even, k <= kClHalo, k <= the rows a block owns,
// so a halo lies in the two neighbouring blocks).  The launch's half-sweeps
// run in phases of k:
//   1. each block takes the halo rows its neighbours pushed at the end of the
//      phase before (two sets of slots, by phase parity);
//   2. k half-sweeps on the window: after half-sweep d (0-based) the window
//      rows 1 + d .. R - 2 - d are exact, so after k of them the block's own
//      rows still are (a trapezoid: the halo rows are recomputed by both
//      neighbours);
//   3. each block pushes its first and last k own rows to the blocks above
//      and below: into their shared memory inside a cluster (distributed
//      shared memory), through a small global buffer with release/acquire
//      sequence flags between clusters;
//   4. a cluster barrier.
// The masks of each half-sweep stream into a ring of shared-memory slabs
// with asynchronous 16-byte copies, up to kClMaxSlabs - 1 half-sweeps ahead.
// Every thread updates the same 1 to 4 window words in each half-sweep
// (those inside its trapezoid), with their offsets worked out once per launch:
// at these sizes a half-sweep is a few hundred instructions per SM, and the
// index arithmetic of a general loop cost as much as the update itself.
// Inside a cluster only the hardware's barriers synchronise.  Between
// clusters a boundary block waits for its neighbour's flag for at most one
// second of the GPU's global timer, then records the failure and carries on,
// so every launch ends and every thread passes the same barriers; the host
// reports the failure.  Each update is the spin logic of row_apply with its
// row's pre-drawn masks, so the results are those of the half-sweep kernels.
// Records (colour 1 of a recorded sweep) count each block's own rows only:
// every bond and spin once.
#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <algorithm>

#include "ising_cluster.cuh"
#include "ising_device.cuh"
#include "ising_internal.h"

namespace cg = cooperative_groups;

namespace ising {
namespace {

constexpr int kClThreads = 1024;           // most threads of a block
constexpr size_t kClSmemMax = 220 * 1024;   // dynamic shared memory of a block
constexpr int kClHalo = 12;                 // most half-sweeps per phase
constexpr int kClMaxSlabs = 8;              // mask slabs where they fit: staged up to 7 half-sweeps ahead

struct ClusterArgs {
    uint64_t* w[2];             // the lattice's colour arrays, L x P words each
    Geom g;
    int k;                      // half-sweeps per phase = halo rows
    int q;                      // mask slabs in shared memory (2 or kClMaxSlabs): masks staged q - 1 half-sweeps ahead
    int nsweeps;                // sweeps of this launch
    int rmax;                   // window rows the shared memory holds (largest share of rows + 2 k)
    const uint64_t* masks;      // masks[(h * L + i) * P + w]: half-sweep h = 2 j + c of the launch, row i, word w
    int64_t s0;                 // the launch runs sweeps s0 + 1 .. s0 + nsweeps of the call
    int64_t every;              // record after sweeps s with s % every == 0 (0: none)
    unsigned long long* counts; // count slots (32 per record); record r of the call -> slot r
    uint32_t all0, all1;        // "always" masks (threshold 2^32)
    int G;                      // clusters of the launch: blocks g C .. g C + C - 1 form cluster g
    uint64_t* xbuf;             // G > 1: halo rows between clusters, [boundary][dir][parity][colour], k x P words
    unsigned long long* xflag;  // G > 1: [boundary][dir] sequence flags
    unsigned long long xseq;    // push m of this launch sets its flags to xseq + m + 1
    unsigned long long xwait;   // added to the values the receives wait for (0; a test stalls with more)
    unsigned int* xerr;         // set to 1 when a wait for a flag gives up
    unsigned int* gate;         // G > 1: the words the blocks agree through (cl_count_in, cl_decide)
    unsigned int gate_blocks;   // blocks that must have counted in (the launch's; one more in a test)
    unsigned int piece;         // the launch's piece of the call
};

// A window word a thread updates in every half-sweep whose rows include its
// row, with what the two colours need worked out once per launch.  The
// neighbour to the side of a site of colour C in global row i is at m - 1
// when (i + C) is even, else m + 1; its word is the next one to the left or
// right, wrapped around the row, whose edge field comes in with a shift of
// 60 bits, or 3 (rlast - 1) across the wrap.
struct Slot {
    uint32_t o;      // lr * P + w (window row lr, word w): the word in the own-colour, other-colour and
                     // mask arrays; ~0u: no word
    uint32_t so;     // the side word's offset for colour 0 (bits 0..15) and colour 1 (16..31)
    uint32_t bits;   // side shift for colour 0 (bits 0..6) and 1 (8..14); colour 0 takes the left
                     // neighbour (16); last word of the row (17); an own row of the block (18)
};

// One update of colour C: the spin logic of row_apply with the packed masks
// p (r < thr1 at bit 3k, r < thr0 at bit 3k + 1, each already set where its
// threshold is 2^32, and zero on the dead fields of a row's last word)
// staged in msk.  Off the spin bits and on dead fields `accept` is then
// zero or masked by kSpinBits: of the four neighbours only h1 can be nonzero
// on a dead field, so there a < 2 and the zero masks decide.  RECORD adds
// the row's anti-aligned bonds and up spins over the live fields.
template <int C, bool RECORD>
__device__ __forceinline__ void cl_update(uint64_t* own, const uint64_t* other, const uint64_t* msk, uint32_t P,
                                          const Slot& sl, uint64_t live_last, uint64_t n, uint32_t& anti,
                                          uint32_t& up)
{
    const uint32_t o = sl.o;
    const bool left = ((sl.bits >> 16) & 1u) != (uint32_t)C;
    const uint32_t so = C == 0 ? (sl.so & 0xffffu) : (sl.so >> 16);
    const uint32_t sh = (sl.bits >> (8 * C)) & 0x7fu;
    const uint64_t s = word_ld<false>(own, o, n, __LINE__);
    const uint64_t u = word_ld<false>(other, o - P, n, __LINE__);
    const uint64_t d = word_ld<false>(other, o + P, n, __LINE__);
    const uint64_t h0 = word_ld<false>(other, o, n, __LINE__);
    const uint64_t side = word_ld<false>(other, so, n, __LINE__);
    const uint64_t p = word_ld<false>(msk, o, n, __LINE__);
    const uint64_t h1 = left ? ((h0 << 3) | (side >> sh)) : ((h0 >> 3) | (side << sh));
    const uint64_t x1 = s ^ u, x2 = s ^ d, x3 = s ^ h0, x4 = s ^ h1;
    const uint64_t any = x1 | x2 | x3 | x4;
    const uint64_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
    const uint64_t accept = ge2 | (any & p) | (~any & (p >> 1));
    const uint64_t s_new = s ^ (accept & kSpinBits);
    word_st(own, o, s_new, n, __LINE__);
    if (RECORD) {
        const uint64_t live = (sl.bits & (1u << 17)) ? live_last : kSpinBits;
        anti += __popcll((s_new ^ u) & live) + __popcll((s_new ^ d) & live) + __popcll((s_new ^ h0) & live)
              + __popcll((s_new ^ h1) & live);
        up += __popcll(s_new & live) + __popcll(h0 & live);
    }
}

// One half-sweep of colour C on window rows lo .. hi: each thread updates
// those of its NS slots that lie there (words lo P .. (hi + 1) P - 1).
// RECORD counts the block's own rows into the count slots `counts`.
template <int C, bool RECORD, int NS>
__device__ __forceinline__ void cl_half_sweep(uint64_t* own, const uint64_t* other, const uint64_t* msk, uint32_t P,
                                              const Slot (&slot)[NS], int lo, int hi, uint64_t live_last,
                                              uint64_t n, unsigned long long* counts)
{
    uint32_t anti = 0, up = 0;
    const uint32_t first = (uint32_t)lo * P, span = (uint32_t)(hi - lo + 1) * P;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (slot[j].o - first < span) {
            if (RECORD && (slot[j].bits & (1u << 18)))
                cl_update<C, true>(own, other, msk, P, slot[j], live_last, n, anti, up);
            else
                cl_update<C, false>(own, other, msk, P, slot[j], live_last, n, anti, up);
        }
    }
    if (RECORD) block_add_counts(counts + 2 * (blockIdx.x % kCountSlots), anti, up);
}

// NS: window words per thread (the block has ceil(words / NS) threads,
// rounded up to whole warps).  DEEP: kClMaxSlabs mask slabs, else 2.
// MULTI: several clusters (G > 1), with the halo exchange between them;
// without it the form has no code for that exchange.
template <int NS, bool DEEP, bool MULTI>
__global__ void __launch_bounds__(NS == 3 ? 768 : kClThreads, 1)
cluster_sweeps_kernel(ClusterArgs a)
{
    extern __shared__ __align__(16) uint64_t smem[];
    // the next piece's mask draw (launched with programmatic stream
    // serialization) may start now, on the SMs this cluster leaves free
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int Q = DEEP ? kClMaxSlabs : 2;
    static_assert((Q & (Q - 1)) == 0, "the mask ring's indices wrap by masking");
    cg::cluster_group cluster = cg::this_cluster();
    const Geom& g = a.g;
    const int T = blockDim.x;
    const int C = (int)cluster.num_blocks(), b = (int)cluster.block_rank();
    const int k = a.k;
    // the launch's G C blocks own consecutive row bands: block B = gc C + b
    const int G = a.G, gc = (int)blockIdx.x / C, NB = G * C, B = gc * C + b;
    // several clusters: count in (a launch after a piece that gave up does nothing)
    if (__builtin_expect(MULTI && !(NS == 1 ? cl_count_in(a.gate, a.piece) : cl_count_in_call(a.gate, a.piece)), 0))
        return;
    // every block of the cluster has started before any block writes into
    // another's shared memory: arrive now, wait just before the first push
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    auto row0 = [&](int blk) { return (int)((long long)blk * g.L / NB); };
    const int r0 = row0(B), r1 = row0(B + 1), S = r1 - r0, R = S + 2 * k;
    const int bp = (b + C - 1) % C, bn = (b + 1) % C;                   // the blocks above and below in the cluster
    // with G > 1 a cluster's first block takes its upper halo from the last
    // block of the cluster above (boundary bd_up, through global memory), its
    // last block the lower halo from the first block of the cluster below
    const bool up_remote = MULTI && b == 0, dn_remote = MULTI && b == C - 1;
    const int bd_up = (gc + G - 1) % G, bd_dn = gc;
    const int top = r0 - k;                                            // global row of window row 0 (mod L)
    const uint32_t P = (uint32_t)g.P;
    const uint64_t n = (uint64_t)a.rmax * P;
    uint64_t* win[2] = {smem, smem + n};
    uint64_t* msk = smem + 2 * n;                                       // Q slabs of n words
    const int pairs = g.P / 2;
    const uint32_t sh_wrap = 3u * (uint32_t)(g.rlast - 1);
    // slots: window words e = t + j T of rows 1 .. R - 2 in steps of the
    // pitch P (a padding word W .. P - 1 has no update: a warp's loads stay
    // on consecutive words, without bank conflicts), and the mask copies (16
    // bytes, word pairs) of the same rows
    Slot slot[NS];
    uint32_t cdst[NS], csrc[NS];
    const uint32_t smem_sh = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t msk_sh = (uint32_t)__cvta_generic_to_shared(msk);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int e = threadIdx.x + j * T;
        const int lr = 1 + e / g.P, w = e % g.P;
        const bool first = w == 0, last = w == g.W - 1;
        const bool left0 = ((top + lr) & 1) == 0;      // colour 0 at (i + 0) even
        // left neighbour: word w - 1 (wrapped), right: w + 1 (wrapped); the
        // window's words fit 16 bits (fewer than 220 KB / 8)
        const uint32_t row = (uint32_t)lr * P;
        const uint32_t sl = row + (uint32_t)(first ? g.W - 1 : w - 1), sr = row + (uint32_t)(last ? 0 : w + 1);
        const uint32_t shl = first ? sh_wrap : 60u, shr = last ? sh_wrap : 60u;
        slot[j].o = lr <= R - 2 && w < g.W ? row + (uint32_t)w : ~0u;
        slot[j].so = ((left0 ? sl : sr) & 0xffffu) | ((left0 ? sr : sl) << 16);
        slot[j].bits = (left0 ? shl : shr) | ((left0 ? shr : shl) << 8) | (left0 ? 1u << 16 : 0u) |
                       (last ? 1u << 17 : 0u) | ((lr >= k && lr < R - k) ? 1u << 18 : 0u);
        const int cr = 1 + e / pairs, cp = e % pairs;
        cdst[j] = cr <= R - 2 ? msk_sh + 8u * ((uint32_t)cr * P + 2u * (uint32_t)cp) : ~0u;   // in slab 0
        csrc[j] = (uint32_t)wrap_index(top + cr, g.L) * P + 2u * (uint32_t)cp;
    }
    const uint64_t live_last = live_mask(g, g.W - 1);
    const int total = 2 * a.nsweeps;
    const size_t plane = (size_t)g.L * P;                               // one half-sweep's masks
    const uint64_t mask_words = (uint64_t)total * plane;                // the launch's mask array
    // masks of the next half-sweep to stage (number `next`) for window rows
    // 1 .. R - 2 into slab `put` (one copy group per half-sweep, empty past
    // the end)
    int next = 0, put = 0;
    const uint64_t smem_words = (uint64_t)(2 + Q) * n + 8 * (uint64_t)k * P;
    const uint32_t slab_bytes = (uint32_t)(n * sizeof(uint64_t));
    const uint64_t* next_src = a.masks;
    auto stage = [&]() {
        if (next < total) {
            const uint32_t off = (uint32_t)put * slab_bytes;
#pragma unroll
            for (int j = 0; j < NS; ++j)
                if (cdst[j] != ~0u)
                    cl_copy_pair(cdst[j] + off, smem_sh, smem_words, next_src + csrc[j], a.masks, mask_words,
                                 __LINE__);
        }
        cl_commit();
        ++next;
        next_src += plane;
        put = (put + 1) & (Q - 1);
    };
    // halo rows: receive slots rb(par, c, 0) for the k rows above the block's
    // own (the last own rows of the block above), rb(par, c, 1) for the k rows
    // below; two sets (par), used by alternate phases
    const int kP = k * (int)P;
    auto rb = [&](uint64_t* base, int par, int c, int dir) { return base + (size_t)((par * 2 + c) * 2 + dir) * kP; };
    uint64_t* recv = msk + (size_t)Q * n;
    // the global slots between clusters: dir 0 carries the last k own rows of
    // cluster bd's last block down to the first block of cluster bd + 1, dir 1
    // the first k own rows of that block up
    auto xs = [&](int bd, int dir, int par, int c) {
        return a.xbuf + (size_t)(((bd * 2 + dir) * 2 + par) * 2 + c) * kP;
    };
    // push m (m = 0 before the first phase, m = p + 1 after phase p): a
    // block's first k own rows go to the slots below of the block above, its
    // last k own rows to the slots above of the block below
    auto push = [&](int par, int m) {
        uint64_t* up_recv = up_remote ? nullptr : cluster.map_shared_rank(recv, bp);
        uint64_t* dn_recv = dn_remote ? nullptr : cluster.map_shared_rank(recv, bn);
        for (int c = 0; c < 2; ++c) {
            uint64_t* to_up = up_remote ? xs(bd_up, 1, par, c) : rb(up_recv, par, c, 1);
            uint64_t* to_dn = dn_remote ? xs(bd_dn, 0, par, c) : rb(dn_recv, par, c, 0);
            for (int idx = threadIdx.x; idx < kP; idx += T) {
                word_st(to_up, idx, word_ld<false>(win[c], (uint64_t)k * P + idx, n, __LINE__), kP, __LINE__);
                word_st(to_dn, idx, word_ld<false>(win[c], (uint64_t)S * P + idx, n, __LINE__), kP, __LINE__);
            }
        }
        if (up_remote || dn_remote) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                if (up_remote) cl_flag_release(a.xflag + bd_up * 2 + 1, a.xseq + m + 1);
                if (dn_remote) cl_flag_release(a.xflag + bd_dn * 2 + 0, a.xseq + m + 1);
            }
        }
    };
    // the halos of phase p (push p of the neighbours)
    auto receive = [&](int par, int p) {
        if (up_remote || dn_remote) {
            if (threadIdx.x == 0) {
                if (up_remote) cl_wait_flag(a.xflag + bd_up * 2 + 0, a.xseq + a.xwait + p + 1, a.xerr);
                if (dn_remote) cl_wait_flag(a.xflag + bd_dn * 2 + 1, a.xseq + a.xwait + p + 1, a.xerr);
            }
            __syncthreads();
        }
        for (int c = 0; c < 2; ++c) {
            const uint64_t* from_up = up_remote ? xs(bd_up, 0, par, c) : rb(recv, par, c, 0);
            const uint64_t* from_dn = dn_remote ? xs(bd_dn, 1, par, c) : rb(recv, par, c, 1);
            for (int idx = threadIdx.x; idx < kP; idx += T) {
                const uint64_t vu = up_remote ? __ldcg(from_up + idx) : word_ld<false>(from_up, idx, kP, __LINE__);
                const uint64_t vd = dn_remote ? __ldcg(from_dn + idx) : word_ld<false>(from_dn, idx, kP, __LINE__);
                word_st(win[c], idx, vu, n, __LINE__);
                word_st(win[c], (uint64_t)(k + S) * P + idx, vd, n, __LINE__);
            }
        }
    };
    // own rows of both colours, from the lattice, to window rows k .. k + S - 1
    for (int c = 0; c < 2; ++c)
        for (int e = threadIdx.x; e < S * pairs; e += T) {
            const int r = e / pairs, cp = e - r * pairs;
            cl_copy_pair(smem_sh + 8u * (uint32_t)(c * n + (size_t)(k + r) * P + 2 * cp), smem_sh, smem_words,
                         a.w[c] + (size_t)(r0 + r) * P + 2 * cp, a.w[c], lattice_words(g), __LINE__);
        }
    cl_commit();
    cl_wait<0>();
    __syncthreads();
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    push(0, 0);
#pragma unroll
    for (int h = 0; h < Q - 1; ++h) stage();
    cluster.sync();          // the first phase's halos have arrived
    int use = 0;             // slab of the current half-sweep
    // before a half-sweep: its slab staged, the previous half-sweep done (its
    // rows final, its slab free for the copies of half-sweep h + Q - 1, which
    // follow the update)
    auto begin = [&]() {
        cl_wait<Q - 2>();
        __syncthreads();
        const uint64_t* m = msk + (size_t)use * n;
        use = (use + 1) & (Q - 1);
        return m;
    };
    // records: sweep j of the launch (1-based) is sweep s0 + j of the call;
    // the next recorded one, rec_j (past nsweeps: none), and its count slot
    int j = 0, rec_j = a.nsweeps + 1;
    unsigned long long* rec_counts = nullptr;
    if (a.every > 0) {
        const int64_t first = (a.s0 / a.every + 1) * a.every;          // first recorded sweep of the call > s0
        if (first - a.s0 <= a.nsweeps) {
            rec_j = (int)(first - a.s0);
            rec_counts = a.counts + (size_t)(first / a.every - 1) * 2 * kCountSlots;
        }
    }
    int par = 0, phase = 0;
    for (int hs0 = 0; hs0 < total; hs0 += k, ++phase) {
        const int kk = min(k, total - hs0);                             // even: phases start with colour 0
        receive(par, phase);  // into the halo rows (ordered before the updates by begin's barrier)
        for (int d = 0; d < kk; d += 2) {
            const uint64_t* m0 = begin();
            cl_half_sweep<0, false, NS>(win[0], win[1], m0, P, slot, 1 + d, R - 2 - d, live_last, n, nullptr);
            stage();
            const uint64_t* m1 = begin();
            if (++j == rec_j) {
                cl_half_sweep<1, true, NS>(win[1], win[0], m1, P, slot, 2 + d, R - 3 - d, live_last, n,
                                           rec_counts);
                rec_counts += 2 * kCountSlots;
                rec_j = a.every <= a.nsweeps - j ? j + (int)a.every : a.nsweeps + 1;
            } else {
                cl_half_sweep<1, false, NS>(win[1], win[0], m1, P, slot, 2 + d, R - 3 - d, live_last, n, nullptr);
            }
            stage();
        }
        par ^= 1;
        if (hs0 + k < total) {
            __syncthreads();     // own rows final for this phase
            push(par, phase + 1);
        }
        // the next phase's halos have arrived; the slots the next pushes write
        // were read at the start of this phase; after the last phase: no block
        // leaves while another may still write its shared memory
        cluster.sync();
    }
    // own rows back to the lattice, with several clusters only if every block
    // of the launch was resident (otherwise none writes)
    cl_wait<0>();
    if (__builtin_expect(MULTI && !(NS == 1 ? cl_decide(a.gate, a.gate_blocks, a.piece)
                                            : cl_decide_call(a.gate, a.gate_blocks, a.piece)), 0))
        return;
    for (int c = 0; c < 2; ++c)
        for (int idx = threadIdx.x; idx < S * (int)P; idx += T)
            word_st(a.w[c], (uint64_t)r0 * P + idx, word_ld<false>(win[c], (uint64_t)k * P + idx, n, __LINE__),
                    lattice_words(g), __LINE__);
}

// Masks of sweeps j = 0 .. nsweeps-1 after sweep (t_base ? *t_base : 0) + t0:
// one thread per (sweep, colour, item) draws them with item_masks_thread (the
// draws of sweep_rows) and writes them row-major, masks[((j * 2 + c) * L + i)
// * P + w], with the bits of a threshold of 2^32 set and those of the dead
// fields of a row's last word cleared.
template <int ROUNDS>
__global__ void __launch_bounds__(128)
cl_mask_draw_kernel(Geom g, SweepArgs a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                    uint64_t* __restrict__ masks)
{
    const int items = ((g.L + 3) / 4) * g.W;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2LL * nsweeps * items) return;
    const int jc = (int)(k / items);
    const int item = (int)(k - (long long)jc * items);
    const int grp = item / g.W;
    const int w = item - grp * g.W;
    const uint64_t t = (t_base ? *t_base : 0) + t0 + (uint64_t)(jc >> 1) + 1;
    uint64_t p[4];
    item_masks_thread<ROUNDS>(g, item, t, jc & 1, a.rk, a.thr0, a.thr1, a.one, p);
    // a threshold of 2^32 accepts always: its bits set here, not in the update
    const uint64_t always = (((uint64_t)a.all1 << 32 | a.all1) & kSpinBits) |
                            ((((uint64_t)a.all0 << 32 | a.all0) & kSpinBits) << 1);
    // the dead fields of a row's last word: both masks zero
    const uint64_t live = live_mask(g, w);
    const uint64_t keep = live | (live << 1);
    uint64_t* out = masks + (size_t)jc * g.L * g.P;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = 4 * grp + e;
        if (i < g.L) out[(size_t)i * g.P + w] = (p[e] | always) & keep;
    }
}

// Both colour windows and q mask slabs (largest share of rows + 2 k rows
// each), and 8 halo receive slots of k rows.
size_t cl_smem_bytes(const Geom& g, int blocks, int k, int q)
{
    const int smax = (g.L + blocks - 1) / blocks;
    return ((size_t)(2 + q) * (smax + 2 * k) + 8 * (size_t)k) * g.P * sizeof(uint64_t);
}

// The forms of the kernel: 1 .. 4 words per thread, 2 or kClMaxSlabs mask
// slabs, one cluster or several.
using ClusterKernel = void (*)(ClusterArgs);
constexpr ClusterKernel kClusterKernels[16] = {
    cluster_sweeps_kernel<1, false, false>, cluster_sweeps_kernel<2, false, false>,
    cluster_sweeps_kernel<3, false, false>, cluster_sweeps_kernel<4, false, false>,
    cluster_sweeps_kernel<1, true, false>,  cluster_sweeps_kernel<2, true, false>,
    cluster_sweeps_kernel<3, true, false>,  cluster_sweeps_kernel<4, true, false>,
    cluster_sweeps_kernel<1, false, true>,  cluster_sweeps_kernel<2, false, true>,
    cluster_sweeps_kernel<3, false, true>,  cluster_sweeps_kernel<4, false, true>,
    cluster_sweeps_kernel<1, true, true>,   cluster_sweeps_kernel<2, true, true>,
    cluster_sweeps_kernel<3, true, true>,   cluster_sweeps_kernel<4, true, true>};

ClusterKernel cluster_kernel(int ns, int q, bool multi)
{
    return kClusterKernels[(multi ? 8 : 0) + (q == kClMaxSlabs ? 4 : 0) + (ns - 1)];
}

// Window words a block takes with at most `ns` words per thread: 1024
// threads for 1, 2 or 4 (64 registers each), 768 for 3 (80 registers).
long long max_words(int ns) { return ns == 3 ? 3 * 768 : (long long)ns * kClThreads; }

// Clusters of the largest size that can be resident at once (set by
// probe_max_cluster).
int g_max_active = 0;

int probe_max_cluster()
{
    for (ClusterKernel kern : kClusterKernels) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmemMax) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.dynamicSmemBytes = kClSmemMax;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        bool ok = true;
        int active = 1 << 30;
        for (int i = 0; i < 16; ++i) {                // form i: (i % 4) + 1 words per thread
            cfg.blockDim = dim3(i % 4 == 2 ? 768 : kClThreads);
            int nc = 0;
            ok = ok && cudaOccupancyMaxActiveClusters(&nc, kClusterKernels[i], &cfg) == cudaSuccess && nc >= 1;
            active = std::min(active, nc);
        }
        if (ok) {
            g_max_active = active;
            return c;
        }
        cudaGetLastError();
    }
    return 0;
}

}  // namespace

// Cluster size, phase length, mask slabs and words per thread for side L:
// 16 blocks if the device runs such a cluster, else 8; k = the most
// half-sweeps per phase (even, <= kClHalo, <= the fewest rows a block owns)
// whose window and kClMaxSlabs mask slabs fit in shared memory (else two
// slabs), with at most 3 window words per thread (1024 threads for 1 or 2,
// 768 for 3) where some k allows it, else 4.  Measured on GB300 (sweeps
// without records, spin-updates/ns, by k = 4 / 8 / 12): L = 296: 77 / 105 /
// 115, L = 512: 170 / 199 / 210, L = 1008: 357 / 394 / 403 (threads over
// the W live words of a row then; over the pitch since, which gave L = 512:
// 215, L = 1008: 416 at k = 12).  3 words per thread against the plan with
// at most 2: L = 1080: 478 (k = 10) against 463 (k = 6); L = 1100: 465
// (k = 6) against 367 (k = 2); 4 words per thread spill registers (L = 1200:
// 297).  Returns false if no such launch exists (a lattice too large or too
// small).
int cluster_max_active()
{
    static const int max_cluster = probe_max_cluster();   // per process, set once
    return max_cluster == 0 ? 0 : g_max_active;
}

bool cluster_plan(const Geom& g, int clusters, ClusterPlan* plan)
{
    static const int max_cluster = probe_max_cluster();   // per process, set once
    if (max_cluster == 0 || clusters < 1 || clusters > g_max_active) return false;
    const int c = max_cluster, nb = clusters * c;         // cluster size, blocks of the launch
    const int fewest = g.L / nb;
    for (int most : {3, 4}) {
        for (int q : {kClMaxSlabs, 2}) {
            for (int kk = std::min(kClHalo, fewest) & ~1; kk >= 2; kk -= 2) {
                if (cl_smem_bytes(g, nb, kk, q) > kClSmemMax) continue;
                const long long words = (long long)((g.L + nb - 1) / nb + 2 * kk - 2) * g.P;
                if (words > max_words(most)) continue;
                const int ns = words <= kClThreads ? 1 : (words <= 2 * kClThreads ? 2 : (words <= max_words(3) ? 3 : 4));
                plan->blocks = c;
                plan->k = kk;
                plan->q = q;
                plan->ns = ns;
                plan->threads = (int)(((words + ns - 1) / ns + 31) / 32 * 32);
                plan->clusters = clusters;
                return true;
            }
        }
    }
    return false;
}

size_t cl_exchange_words(const Geom& g, const ClusterPlan& plan)
{
    return (size_t)plan.clusters * 2 * 2 * 2 * plan.k * g.P;     // [boundary][dir][parity][colour] k x P
}

unsigned long long cl_exchange_seqs(const ClusterPlan& plan, int nsweeps)
{
    return (unsigned long long)((2 * nsweeps + plan.k - 1) / plan.k) + 1;   // pushes of a launch, + 1
}

size_t cl_mask_bytes_per_sweep(const Geom& g) { return 2 * (size_t)g.L * g.P * sizeof(uint64_t); }

cudaError_t launch_cl_mask_draw(const Geom& g, const SweepArgs& a, const uint64_t* t_base, uint64_t t0, int nsweeps,
                                uint64_t* masks, bool overlap, cudaStream_t s)
{
    const long long threads = 2LL * nsweeps * (((g.L + 3) / 4) * g.W);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((threads + 127) / 128));
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    return a.rounds == 7 ? cudaLaunchKernelEx(&cfg, cl_mask_draw_kernel<7>, g, a, t_base, t0, nsweeps, masks)
                         : cudaLaunchKernelEx(&cfg, cl_mask_draw_kernel<10>, g, a, t_base, t0, nsweeps, masks);
}

cudaError_t launch_cluster_sweeps(uint64_t* w0, uint64_t* w1, const Geom& g, const SweepArgs& a,
                                  const ClusterPlan& plan, int nsweeps, const uint64_t* masks, int64_t s0,
                                  int64_t every, const ClusterExchange& x, cudaStream_t s)
{
    const int nb = plan.clusters * plan.blocks;
    ClusterArgs ca;
    ca.w[0] = w0;
    ca.w[1] = w1;
    ca.g = g;
    ca.k = plan.k;
    ca.q = plan.q;
    ca.nsweeps = nsweeps;
    ca.rmax = (g.L + nb - 1) / nb + 2 * plan.k;
    ca.masks = masks;
    ca.s0 = s0;
    ca.every = every;
    ca.counts = a.counts;
    ca.all0 = a.all0;
    ca.all1 = a.all1;
    ca.G = plan.clusters;
    ca.xbuf = x.buf;
    ca.xflag = x.flags;
    ca.xseq = x.seq;
    ca.xwait = x.wait_add;
    ca.xerr = x.err;
    ca.gate = x.gate;
    ca.gate_blocks = (unsigned int)(nb) + x.absent;
    ca.piece = x.piece;
    if (plan.clusters > 1 && (!x.buf || !x.flags || !x.err || !x.gate)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = cl_smem_bytes(g, nb, plan.k, plan.q);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.blocks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_kernel(plan.ns, plan.q, plan.clusters > 1), ca);
}

}  // namespace ising

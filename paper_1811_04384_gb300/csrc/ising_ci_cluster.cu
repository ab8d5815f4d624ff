// Cluster-resident temporal blocking in the paper's column-interleaved
// layout (Sec. 3): the form of ising_cluster.cu for N x L words, mid-size
// lattices (L a multiple of 84 up to about 2600).
//
// Word S(I, J) holds s(I + kN, J) in field k and has colour (I + J) & 1.  A
// half-sweep's neighbours of a word are the words left and right in its row
// and above and below in its column, rotated by one field across the top
// and bottom word rows (the paper's boundary rule).  So the lattice splits
// by columns: block B of the launch's G thread-block clusters owns word
// columns c0(B) .. c0(B + 1) - 1 (multiples of 4) of all N word rows and
// keeps them in shared memory for a piece of up to 256 sweeps, in a window
// with k halo columns on each side (k a multiple of 4).  Phases of k
// half-sweeps shrink the valid columns by one per half-sweep (a trapezoid);
// at the end of a phase each block pushes its first and last k own columns
// into the receive slots of its left and right neighbours (distributed shared
// memory inside a cluster, the global buffer and flags of ising_cluster.cu
// between clusters, two sets by phase parity) and the blocks of a cluster
// pass one hardware cluster barrier.
//
// The window is kept split by column parity: E holds the even window
// columns, O the odd ones, pair p = columns 2p, 2p + 1.  In row I the word
// of colour C of pair p is in E when (I + C) is even, else in O; its
// up / down neighbours are in the same array, its left / right neighbours in
// the other at pairs p - 1, p or p, p + 1.  So every load of a warp over
// consecutive pairs falls on consecutive words.  The accept masks, drawn
// beforehand on the SMs the cluster leaves free (ci_masks, the draws of the
// other interleaved kernels), stream into a ring of shared-memory slabs
// indexed like the pairs.  The update is Eq. 3 summed bitwise, as in the
// row-packed kernels: the decisions of ci_half_sweep_apply_kernel's 3-bit
// field sums, so the results equal every other path's.
#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <algorithm>

#include "ising_cluster.cuh"
#include "ising_interleaved.cuh"
#include "ising_interleaved.h"
#include "ising_internal.h"

namespace cg = cooperative_groups;

namespace ising {
namespace {

constexpr int kCiThreads = 1024;           // most threads of a block
constexpr size_t kCiSmemMax = 220 * 1024;   // dynamic shared memory of a block
constexpr int kCiHalo = 12;                 // most half-sweeps per phase (a multiple of 4)
constexpr int kCiMaxSlabs = 8;              // mask slabs where they fit

struct CiClusterArgs {
    uint64_t* S;                // the lattice, N x L words
    int L, N;
    int k;                      // half-sweeps per phase = halo columns
    int nsweeps;                // sweeps of this launch
    int wpm;                    // pairs per window row (the widest block's columns + 2 k, halved)
    const uint64_t* masks;      // masks[(h * N + I) * L/2 + m]: half-sweep h, word row I, column pair m
    int64_t s0;                 // the launch runs sweeps s0 + 1 .. s0 + nsweeps of the call
    int64_t every;              // record after sweeps s with s % every == 0 (0: none)
    unsigned long long* counts; // count slots (32 per record); record r of the call -> slot r
    int G;                      // clusters of the launch: blocks g C .. g C + C - 1 form cluster g
    uint64_t* xbuf;             // G > 1: halo columns between clusters, [boundary][dir][parity][array], N x k/2 words
    unsigned long long* xflag;  // G > 1: [boundary][dir] sequence flags
    unsigned long long xseq;    // push m of this launch sets its flags to xseq + m + 1
    unsigned long long xwait;   // added to the values the receives wait for (0; a test stalls with more)
    unsigned int* xerr;         // set to 1 when a wait for a flag gives up
    unsigned int* gate;         // G > 1: the words the blocks agree through (cl_count_in, cl_decide)
    unsigned int gate_blocks;   // blocks that must have counted in (the launch's; one more in a test)
    unsigned int piece;         // the launch's piece of the call
};

// First word column of block b of a cluster of C: a multiple of 4.
__host__ __device__ __forceinline__ int ci_col0(int b, int C, int L)
{
    return 4 * (int)((long long)b * (L / 4) / C);
}

// A window pair a thread updates (the word of the half-sweep's colour in it)
// in every half-sweep whose columns include that word.
struct CiSlot {
    uint32_t o;      // I * wpm + p: the pair in E, O and the mask slabs; ~0u: none
    uint32_t bits;   // window column of the colour-0 word (bits 0..15); colour 0's word in O (16);
                     // top word row (17); bottom word row (18); an own column pair of the block (19)
};

// One update of colour C (Eq. 3): s, its four neighbours and
// the packed masks p (r < thr1 at bit 3k, r < thr0 at 3k + 1, set where the
// threshold is 2^32).  RECORD adds the word's anti-aligned bonds and the up
// spins of its column pair.
template <int C, bool RECORD>
__device__ __forceinline__ void ci_cl_update(uint64_t* E, const uint64_t* msk, uint32_t wpm, uint32_t wrap,
                                             uint64_t nw, const CiSlot& sl, uint32_t& anti, uint32_t& up)
{
    const uint32_t o = sl.o;
    const uint32_t par = ((sl.bits >> 16) & 1u) ^ (uint32_t)C;       // 0: the word is in E, 1: in O
    uint64_t* own = E + (size_t)par * nw;
    const uint64_t* oth = E + (size_t)(par ^ 1u) * nw;
    const uint64_t s = word_ld<false>(own, o, nw, __LINE__);
    const bool top = (sl.bits >> 17) & 1u, bottom = (sl.bits >> 18) & 1u;
    const uint64_t wu = word_ld<false>(own, top ? o + wrap : o - wpm, nw, __LINE__);
    const uint64_t wd = word_ld<false>(own, bottom ? o - wrap : o + wpm, nw, __LINE__);
    const uint64_t xu = top ? rotate_up(wu) : wu;
    const uint64_t xd = bottom ? rotate_down(wd) : wd;
    const uint64_t xl = word_ld<false>(oth, o - 1u + par, nw, __LINE__);
    const uint64_t xr = word_ld<false>(oth, o + par, nw, __LINE__);
    const uint64_t p = word_ld<false>(msk, o, nw, __LINE__);
    // Eq. 3 summed bitwise (as the row-packed kernels do): with x_n = s ^ n
    // the field's spin bit of x_n is set iff neighbour n is anti-aligned;
    // a >= 1 is their OR, a >= 2 that two of them are set.  The same
    // decisions as the carry-free 3-bit field sum of the other interleaved
    // kernels, in fewer instructions.
    const uint64_t x1 = s ^ xu, x2 = s ^ xd, x3 = s ^ xl, x4 = s ^ xr;
    const uint64_t any = x1 | x2 | x3 | x4;
    const uint64_t ge2 = (x1 & x2) | (x3 & x4) | ((x1 ^ x2) & (x3 ^ x4));
    const uint64_t accept = ge2 | (any & p) | (~any & (p >> 1));
    const uint64_t sn = s ^ (accept & kAllFields);
    word_st(own, o, sn, nw, __LINE__);
    if (RECORD) {
        const uint64_t pair_other = par ? xl : xr;       // the pair's other word
        anti += __popcll(sn ^ xu) + __popcll(sn ^ xd) + __popcll(sn ^ xl) + __popcll(sn ^ xr);
        up += __popcll(sn) + __popcll(pair_other);
    }
}

// One half-sweep of colour C on window columns lo .. hi.
template <int C, bool RECORD, int NS>
__device__ __forceinline__ void ci_cl_half_sweep(uint64_t* E, const uint64_t* msk, uint32_t wpm, uint32_t wrap,
                                                 uint64_t nw, const CiSlot (&slot)[NS], int lo, int hi,
                                                 unsigned long long* counts)
{
    uint32_t anti = 0, up = 0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int w = (int)(slot[j].bits & 0xffffu) ^ C;              // the colour-C word's window column
        if (slot[j].o != ~0u && w >= lo && w <= hi) {
            if (RECORD && (slot[j].bits & (1u << 19)))
                ci_cl_update<C, true>(E, msk, wpm, wrap, nw, slot[j], anti, up);
            else
                ci_cl_update<C, false>(E, msk, wpm, wrap, nw, slot[j], anti, up);
        }
    }
    if (RECORD) block_add_counts(counts + 2 * (blockIdx.x % kCountSlots), anti, up);
}

// NS: window pairs per thread; DEEP: kCiMaxSlabs mask slabs, else 2;
// MULTI: several clusters, whose boundary blocks pass their halo columns
// through global memory (as in cluster_sweeps_kernel).
template <int NS, bool DEEP, bool MULTI>
__global__ void __launch_bounds__(NS == 3 ? 768 : kCiThreads, 1)
ci_cluster_sweeps_kernel(CiClusterArgs a)
{
    extern __shared__ __align__(16) uint64_t smem[];
    // the next piece's mask draw (launched with programmatic stream
    // serialization) may start now, on the SMs this cluster leaves free
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int Q = DEEP ? kCiMaxSlabs : 2;
    static_assert((Q & (Q - 1)) == 0, "the mask ring's indices wrap by masking");
    cg::cluster_group cluster = cg::this_cluster();
    const int T = blockDim.x;
    const int C = (int)cluster.num_blocks(), b = (int)cluster.block_rank();
    const int L = a.L, N = a.N, k = a.k, kh = k / 2, PL = L / 2;
    // the launch's G C blocks own consecutive column bands: block B = gc C + b
    const int G = a.G, gc = (int)blockIdx.x / C, NB = G * C, B = gc * C + b;
    // several clusters: count in (a launch after a piece that gave up does nothing)
    if (__builtin_expect(MULTI && !(NS == 1 ? cl_count_in(a.gate, a.piece) : cl_count_in_call(a.gate, a.piece)), 0))
        return;
    // every block of the cluster has started before any block writes into
    // another's shared memory: arrive now, wait just before the first push
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    const int c0 = ci_col0(B, NB, L), S = ci_col0(B + 1, NB, L) - c0;  // own columns
    const int bp = (b + C - 1) % C, bn = (b + 1) % C;                  // left and right blocks in the cluster
    // with G > 1 a cluster's first block takes its left halo from the last
    // block of the cluster to its left (boundary bd_l, global memory), its
    // last block the right halo from the first block of the next cluster
    const bool l_remote = MULTI && b == 0, r_remote = MULTI && b == C - 1;
    const int bd_l = (gc + G - 1) % G, bd_r = gc;
    const int Wn = S + 2 * k, Wp = Wn / 2;                               // window columns and pairs
    const uint32_t wpm = (uint32_t)a.wpm;
    const uint64_t nw = (uint64_t)N * wpm;                              // words of E, O, a slab
    uint64_t* E = smem;                                                  // O = E + nw
    uint64_t* msk = smem + 2 * nw;                                       // Q slabs
    uint64_t* recv = msk + (size_t)Q * nw;                               // receive slots
    const int slotw = N * kh;                                            // words of one receive slot
    const uint64_t smem_words = (2 + Q) * nw + 8 * (uint64_t)slotw;
    const uint32_t smem_sh = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t msk_sh = (uint32_t)__cvta_generic_to_shared(msk);
    const int gp0 = c0 / 2 - kh;                                         // global pair of window pair 0 (mod PL)
    const uint32_t wrap = (uint32_t)(N - 1) * wpm;                       // top <-> bottom word row
    // slots: pairs e = t + j T over the rows (I = e / wpm, p = e % wpm), and
    // the mask copies (16 bytes: two pairs) of the same rows
    CiSlot slot[NS];
    uint32_t cdst[NS], csrc[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int e = threadIdx.x + j * T;
        const int I = e / (int)wpm, p = e % (int)wpm;
        const bool valid = I < N && p < Wp;
        const int par0 = I & 1;                                          // colour 0's word: column 2p + par0
        slot[j].o = valid ? (uint32_t)e : ~0u;
        slot[j].bits = (uint32_t)(2 * p + par0) | ((uint32_t)par0 << 16) | (I == 0 ? 1u << 17 : 0u) |
                       (I == N - 1 ? 1u << 18 : 0u) | ((p >= kh && p < kh + S / 2) ? 1u << 19 : 0u);
        const int half = (int)wpm / 2;                                   // copies per window row
        const int cI = e / half, cq = e % half;
        cdst[j] = cI < N && cq < Wp / 2 ? msk_sh + 8u * ((uint32_t)cI * wpm + 2u * (uint32_t)cq) : ~0u;
        csrc[j] = (uint32_t)cI * (uint32_t)PL + (uint32_t)wrap_index(gp0 + 2 * cq, PL);
    }
    const int total = 2 * a.nsweeps;
    const size_t plane = (size_t)N * PL;                                 // one half-sweep's masks
    const uint64_t mask_words = (uint64_t)total * plane;
    const uint32_t slab_bytes = (uint32_t)(nw * sizeof(uint64_t));
    const uint64_t* next_src = a.masks;
    int next = 0, put = 0;
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
    // receive slots: rs(par, dir, arr) holds k/2 pairs of array arr (0: E,
    // 1: O) of all word rows, dir 0 for the block's left halo (the left
    // block's last k own columns), 1 for its right halo; two sets by phase
    auto rs = [&](uint64_t* base, int par, int dir, int arr) {
        return base + (size_t)((par * 2 + dir) * 2 + arr) * slotw;
    };
    // a block's first k own columns (pairs kh .. k - 1) go to the right-halo
    // slots of the left block, its last k (pairs S/2 .. S/2 + kh - 1) to the
    // left-halo slots of the right block
    // the global slots between clusters: dir 0 carries the last k own columns
    // of cluster bd's last block right to the first block of cluster bd + 1,
    // dir 1 the first k own columns of that block left
    auto xs = [&](int bd, int dir, int par, int arr) {
        return a.xbuf + (size_t)(((bd * 2 + dir) * 2 + par) * 2 + arr) * slotw;
    };
    // push m (m = 0 before the first phase, m = p + 1 after phase p)
    auto push = [&](int par, int m) {
        uint64_t* to_left = l_remote ? nullptr : cluster.map_shared_rank(recv, bp);
        uint64_t* to_right = r_remote ? nullptr : cluster.map_shared_rank(recv, bn);
        for (int arr = 0; arr < 2; ++arr) {
            const uint64_t* A = E + (size_t)arr * nw;
            uint64_t* dl = l_remote ? xs(bd_l, 1, par, arr) : rs(to_left, par, 1, arr);
            uint64_t* dr = r_remote ? xs(bd_r, 0, par, arr) : rs(to_right, par, 0, arr);
            for (int idx = threadIdx.x; idx < slotw; idx += T) {
                const int I = idx / kh, x = idx - I * kh;
                word_st(dl, idx, word_ld<false>(A, (uint64_t)I * wpm + kh + x, nw, __LINE__), slotw, __LINE__);
                word_st(dr, idx, word_ld<false>(A, (uint64_t)I * wpm + S / 2 + x, nw, __LINE__), slotw, __LINE__);
            }
        }
        if (l_remote || r_remote) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                if (l_remote) cl_flag_release(a.xflag + bd_l * 2 + 1, a.xseq + m + 1);
                if (r_remote) cl_flag_release(a.xflag + bd_r * 2 + 0, a.xseq + m + 1);
            }
        }
    };
    // the halos of phase p (push p of the neighbours)
    auto receive = [&](int par, int p) {
        if (l_remote || r_remote) {
            if (threadIdx.x == 0) {
                if (l_remote) cl_wait_flag(a.xflag + bd_l * 2 + 0, a.xseq + a.xwait + p + 1, a.xerr);
                if (r_remote) cl_wait_flag(a.xflag + bd_r * 2 + 1, a.xseq + a.xwait + p + 1, a.xerr);
            }
            __syncthreads();
        }
        for (int arr = 0; arr < 2; ++arr) {
            uint64_t* A = E + (size_t)arr * nw;
            const uint64_t* fl = l_remote ? xs(bd_l, 0, par, arr) : rs(recv, par, 0, arr);
            const uint64_t* fr = r_remote ? xs(bd_r, 1, par, arr) : rs(recv, par, 1, arr);
            for (int idx = threadIdx.x; idx < slotw; idx += T) {
                const int I = idx / kh, x = idx - I * kh;
                const uint64_t vl = l_remote ? __ldcg(fl + idx) : word_ld<false>(fl, idx, slotw, __LINE__);
                const uint64_t vr = r_remote ? __ldcg(fr + idx) : word_ld<false>(fr, idx, slotw, __LINE__);
                word_st(A, (uint64_t)I * wpm + x, vl, nw, __LINE__);
                word_st(A, (uint64_t)I * wpm + (S + k) / 2 + x, vr, nw, __LINE__);
            }
        }
    };
    // own columns from the lattice: word (I, c0 + x) -> window column k + x
    const uint64_t lattice_n = (uint64_t)N * L;
    for (int e = threadIdx.x; e < N * S; e += T) {
        const int I = e / S, x = e - I * S;
        const int w = k + x;
        word_st(E + (size_t)(w & 1) * nw, (uint64_t)I * wpm + (w >> 1),
                word_ld<false>(a.S, (uint64_t)I * L + c0 + x, lattice_n, __LINE__), nw, __LINE__);
    }
    __syncthreads();
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    push(0, 0);
#pragma unroll
    for (int h = 0; h < Q - 1; ++h) stage();
    cluster.sync();          // the first phase's halos have arrived
    int use = 0;             // slab of the current half-sweep
    auto begin = [&]() {
        cl_wait<Q - 2>();
        __syncthreads();
        const uint64_t* m = msk + (size_t)use * nw;
        use = (use + 1) & (Q - 1);
        return m;
    };
    // records: sweep j of the launch is sweep s0 + j of the call
    int j = 0, rec_j = a.nsweeps + 1;
    unsigned long long* rec_counts = nullptr;
    if (a.every > 0) {
        const int64_t first = (a.s0 / a.every + 1) * a.every;
        if (first - a.s0 <= a.nsweeps) {
            rec_j = (int)(first - a.s0);
            rec_counts = a.counts + (size_t)(first / a.every - 1) * 2 * kCountSlots;
        }
    }
    int par = 0, phase = 0;
    for (int hs0 = 0; hs0 < total; hs0 += k, ++phase) {
        const int kk = min(k, total - hs0);                             // even: phases start with colour 0
        receive(par, phase);
        for (int d = 0; d < kk; d += 2) {
            const uint64_t* m0 = begin();
            ci_cl_half_sweep<0, false, NS>(E, m0, wpm, wrap, nw, slot, 1 + d, Wn - 2 - d, nullptr);
            stage();
            const uint64_t* m1 = begin();
            if (++j == rec_j) {
                ci_cl_half_sweep<1, true, NS>(E, m1, wpm, wrap, nw, slot, 2 + d, Wn - 3 - d, rec_counts);
                rec_counts += 2 * kCountSlots;
                rec_j = a.every <= a.nsweeps - j ? j + (int)a.every : a.nsweeps + 1;
            } else {
                ci_cl_half_sweep<1, false, NS>(E, m1, wpm, wrap, nw, slot, 2 + d, Wn - 3 - d, nullptr);
            }
            stage();
        }
        par ^= 1;
        if (hs0 + k < total) {
            __syncthreads();     // own columns final for this phase
            push(par, phase + 1);
        }
        // the next phase's halos have arrived; the slots the next pushes write
        // were read at the start of this phase; after the last phase: no block
        // leaves while another may still write its shared memory
        cluster.sync();
    }
    // own columns back to the lattice, with several clusters only if every
    // block of the launch was resident (otherwise none writes)
    cl_wait<0>();
    if (__builtin_expect(MULTI && !(NS == 1 ? cl_decide(a.gate, a.gate_blocks, a.piece)
                                            : cl_decide_call(a.gate, a.gate_blocks, a.piece)), 0))
        return;
    for (int e = threadIdx.x; e < N * S; e += T) {
        const int I = e / S, x = e - I * S;
        const int w = k + x;
        word_st(a.S, (uint64_t)I * L + c0 + x,
                word_ld<false>(E + (size_t)(w & 1) * nw, (uint64_t)I * wpm + (w >> 1), nw, __LINE__), lattice_n,
                __LINE__);
    }
}

// Masks of sweeps j = 0 .. nsweeps-1 after sweep t0, one thread per (sweep,
// colour, row group q, column pair m) with ci_masks, written as planes:
// masks[((j * 2 + c) * N + 4 q + e) * L/2 + m], with the bits of a
// threshold of 2^32 set.
template <int ROUNDS>
__global__ void __launch_bounds__(128)
ci_cl_mask_draw_kernel(int L, int N, SweepArgs a, uint64_t t0, int nsweeps, uint64_t* __restrict__ masks)
{
    const long long Q4 = N / 4, M = L / 2;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)nsweeps * 2 * Q4 * M) return;
    const int m = (int)(k % M);
    const int q = (int)((k / M) % Q4);
    const int jc = (int)(k / (M * Q4));                 // sweep * 2 + colour
    uint64_t packed[4];
    ci_masks<ROUNDS>(N, q, m, t0 + (uint64_t)(jc >> 1) + 1, jc & 1, a, packed);
    const uint64_t always = (((uint64_t)a.all1 << 32 | a.all1) & kAllFields) |
                            ((((uint64_t)a.all0 << 32 | a.all0) & kAllFields) << 1);
    uint64_t* plane = masks + (size_t)jc * N * M;
#pragma unroll
    for (int e = 0; e < 4; ++e) plane[(size_t)(4 * q + e) * M + m] = packed[e] | always;
}

// The widest block's columns: c0(b + 1) - c0(b) <= 4 ceil((L / 4) / C).
int ci_widest(int L, int C) { return 4 * ((L / 4 + C - 1) / C); }

// E, O and q mask slabs of N x wpm words, and 8 receive slots of N x k / 2.
size_t ci_cl_smem_bytes(int L, int N, int C, int k, int q)
{
    const size_t wpm = (size_t)(ci_widest(L, C) + 2 * k) / 2;
    return ((size_t)(2 + q) * N * wpm + 4 * (size_t)N * k) * sizeof(uint64_t);
}

using CiClusterKernel = void (*)(CiClusterArgs);
constexpr CiClusterKernel kCiClusterKernels[16] = {
    ci_cluster_sweeps_kernel<1, false, false>, ci_cluster_sweeps_kernel<2, false, false>,
    ci_cluster_sweeps_kernel<3, false, false>, ci_cluster_sweeps_kernel<4, false, false>,
    ci_cluster_sweeps_kernel<1, true, false>,  ci_cluster_sweeps_kernel<2, true, false>,
    ci_cluster_sweeps_kernel<3, true, false>,  ci_cluster_sweeps_kernel<4, true, false>,
    ci_cluster_sweeps_kernel<1, false, true>,  ci_cluster_sweeps_kernel<2, false, true>,
    ci_cluster_sweeps_kernel<3, false, true>,  ci_cluster_sweeps_kernel<4, false, true>,
    ci_cluster_sweeps_kernel<1, true, true>,   ci_cluster_sweeps_kernel<2, true, true>,
    ci_cluster_sweeps_kernel<3, true, true>,   ci_cluster_sweeps_kernel<4, true, true>};

CiClusterKernel ci_cluster_kernel(int ns, int q, bool multi)
{
    return kCiClusterKernels[(multi ? 8 : 0) + (q == kCiMaxSlabs ? 4 : 0) + (ns - 1)];
}

// Window words a block takes with at most `ns` words per thread: 1024
// threads for 1, 2 or 4 (64 registers each), 768 for 3 (80 registers).
long long max_words(int ns) { return ns == 3 ? 3 * 768 : (long long)ns * kCiThreads; }

int g_ci_max_active = 0;   // clusters of the largest size resident at once (set by the probe)

int ci_probe_max_cluster()
{
    for (CiClusterKernel kern : kCiClusterKernels) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCiSmemMax) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.dynamicSmemBytes = kCiSmemMax;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        bool ok = true;
        int active = 1 << 30;
        for (int i = 0; i < 16; ++i) {                // form i: (i % 4) + 1 pairs per thread
            cfg.blockDim = dim3(i % 4 == 2 ? 768 : kCiThreads);
            int nc = 0;
            ok = ok && cudaOccupancyMaxActiveClusters(&nc, kCiClusterKernels[i], &cfg) == cudaSuccess && nc >= 1;
            active = std::min(active, nc);
        }
        if (ok) {
            g_ci_max_active = active;
            return c;
        }
        cudaGetLastError();
    }
    return 0;
}

}  // namespace

// Cluster size, phase length (a multiple of 4, <= kCiHalo, <= the fewest
// columns a block owns), mask slabs and pairs per thread for side L, as
// cluster_plan: the largest k whose window, kCiMaxSlabs slabs (else 2) and
// receive slots fit in shared memory with at most 3 pairs per thread where
// some k allows it, else 4 (L = 1008: k = 12 with 3 pairs per thread, 373
// spin-updates/ns, against k = 8 with 2, 367; L = 1092: 3 pairs, 403,
// against 4, 232).  False if L is not a side of the layout or no such launch
// exists.
bool ci_cluster_plan(int L, int clusters, ClusterPlan* plan)
{
    if (!ci_valid_side(L)) return false;
    static const int max_cluster = ci_probe_max_cluster();   // per process, set once
    if (max_cluster == 0 || clusters < 1 || clusters > g_ci_max_active) return false;
    const int c = max_cluster, nb = clusters * c, N = L / 21;         // cluster size, blocks of the launch
    const int fewest = 4 * ((L / 4) / nb), widest = ci_widest(L, nb);
    for (int most : {3, 4}) {
        for (int q : {kCiMaxSlabs, 2}) {
            for (int kk = std::min(kCiHalo, fewest) & ~3; kk >= 4; kk -= 4) {
                if (ci_cl_smem_bytes(L, N, nb, kk, q) > kCiSmemMax) continue;
                const long long words = (long long)N * ((widest + 2 * kk) / 2);
                if (words > max_words(most)) continue;
                const int ns = words <= kCiThreads ? 1 : (words <= 2 * kCiThreads ? 2 : (words <= max_words(3) ? 3 : 4));
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

size_t ci_cl_exchange_words(int L, const ClusterPlan& plan)
{
    return (size_t)plan.clusters * 2 * 2 * 2 * (L / 21) * (plan.k / 2);   // [boundary][dir][parity][array] N x k/2
}

size_t ci_cl_mask_bytes_per_sweep(int L) { return 2 * (size_t)(L / 21) * (L / 2) * sizeof(uint64_t); }

cudaError_t ci_cl_mask_draw(int L, const SweepArgs& a, uint64_t t0, int nsweeps, uint64_t* masks, bool overlap,
                            cudaStream_t s)
{
    const int N = L / 21;
    const long long threads = (long long)nsweeps * 2 * (N / 4) * (L / 2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((threads + 127) / 128));
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    return a.rounds == 7 ? cudaLaunchKernelEx(&cfg, ci_cl_mask_draw_kernel<7>, L, N, a, t0, nsweeps, masks)
                         : cudaLaunchKernelEx(&cfg, ci_cl_mask_draw_kernel<10>, L, N, a, t0, nsweeps, masks);
}

cudaError_t ci_cluster_sweeps(uint64_t* S, int L, const SweepArgs& a, const ClusterPlan& plan, int nsweeps,
                              const uint64_t* masks, int64_t s0, int64_t every, const ClusterExchange& x,
                              cudaStream_t s)
{
    const int nb = plan.clusters * plan.blocks;
    CiClusterArgs ca;
    ca.S = S;
    ca.L = L;
    ca.N = L / 21;
    ca.k = plan.k;
    ca.nsweeps = nsweeps;
    ca.wpm = (ci_widest(L, nb) + 2 * plan.k) / 2;
    ca.masks = masks;
    ca.s0 = s0;
    ca.every = every;
    ca.counts = a.counts;
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
    cfg.dynamicSmemBytes = ci_cl_smem_bytes(L, ca.N, nb, plan.k, plan.q);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.blocks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ci_cluster_kernel(plan.ns, plan.q, plan.clusters > 1), ca);
}

}  // namespace ising

// Helpers of the cluster kernels (ising_cluster.cu, ising_ci_cluster.cu):
// asynchronous 16-byte copies into shared memory, with a range-checked form
// for the checked build, and the flags of the exchanges between clusters.
#pragma once
#include <cstdint>

#include "ising_device.cuh"

namespace ising {
namespace {

// 16 bytes global -> shared (a 32-bit shared-window address), asynchronously,
// through L2.
__device__ __forceinline__ void cl_copy16(uint32_t smem_dst, const void* gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_dst), "l"(gmem_src) : "memory");
}

// cl_copy16 to shared address `dst` from `src`.  In a checked build the
// copy is skipped and recorded (see word_ld) unless both words of the pair
// lie in the `dst_words` words from shared address `dst_base` and in the
// `src_words` words from `src_base`.
__device__ __forceinline__ void cl_copy_pair(uint32_t dst, uint32_t dst_base, uint64_t dst_words, const uint64_t* src,
                                             const uint64_t* src_base, uint64_t src_words, uint32_t line)
{
#ifdef ISING_CHECKED
    if (!check_index((uint64_t)(dst - dst_base) / 8 + 1, dst_words, line) ||
        !check_index((uint64_t)(src - src_base) + 1, src_words, line))
        return;
#else
    (void)dst_base;
    (void)dst_words;
    (void)src_base;
    (void)src_words;
    (void)line;
#endif
    cl_copy16(dst, src);
}

__device__ __forceinline__ void cl_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cl_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ int wrap_index(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

// Sequence flags of the exchanges between clusters (global memory).  The
// writer stores the rows, fences, passes a block barrier, and one thread
// stores the flag with release semantics; the reader's one thread waits for
// it with acquire loads, the block passes a barrier, and its threads read the
// rows past L1 (__ldcg).
__device__ __forceinline__ void cl_flag_release(unsigned long long* f, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(f), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long cl_flag_acquire(const unsigned long long* f)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(f) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long cl_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kClWaitNs = 1000000000ull;   // a wait gives up after one second

__device__ __forceinline__ unsigned int cl_load_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The agreement of a launch with several clusters.  Its boundary blocks
// wait for rows from other clusters, which needs every cluster of the launch
// resident at once; other work on the device (another stream or process) can
// hold SMs so that some are not, and then those waits give up and the rows
// are stale.  So a launch writes its lattice rows back only if all its blocks
// were resident together, and all its blocks agree on that:
//   gate[0..3]  two sets of {blocks counted in, verdict}, used by alternate
//               pieces of a call (both zeroed before the call's first launch);
//   gate[4]     the first piece of the call whose launch gave up (kClNoPiece
//               before it; the launches after it in the call do nothing).
// Every block counts in as it starts (cl_count_in, no wait) and decides at
// its end, before the write-back (cl_decide): it proposes "go" (1) if it sees
// all blocks counted in, else, after kClCheckInNs, "give up" (2).  The first
// proposal written is the verdict every block reads, so the blocks all write
// back or none does; "go" implies that every block had started while the
// proposer ran, so all were resident together.  Normally each block finds
// the count complete at once, and nobody waits.  On "go" block 0 zeroes the
// other set for the next piece (the launch before, which used it, has ended).
// The kernels with more than one word per thread call them through the
// non-inlined forms below: inlined, they cost the 80-register form a spill
// in its loop (3% at L = 2016 on GB300); the one-word form runs faster with
// them inlined (3% at L = 1008).
constexpr unsigned int kClCheckInNs = 100000000u;   // 0.1 s (on the low 32 bits of the global timer)
constexpr unsigned int kClNoPiece = 0xffffffffu;

__device__ __forceinline__ unsigned int cl_globaltimer_lo()
{
    unsigned int t;
    asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
    return t;
}

// Every thread of the block: false if an earlier piece of the call gave up
// (then the block returns at once); else thread 0 has counted the block in.
// Only an earlier piece counts: this launch's own give-up can be written
// while its late clusters start, and the blocks of a cluster must all go on
// or all return (they write into one another's shared memory).
__device__ __forceinline__ bool cl_count_in(unsigned int* gate, unsigned int piece)
{
    int live = 0;
    if (threadIdx.x == 0 && cl_load_acquire(gate + 4) >= piece) {
        atomicAdd(gate + 2 * (piece & 1u), 1u);
        live = 1;
    }
    return __syncthreads_or(live) != 0;
}

// Every thread of the block, at its end: true if the launch writes back.
__device__ __forceinline__ bool cl_decide(unsigned int* gate, unsigned int blocks, unsigned int piece)
{
    int go = 0;
    if (threadIdx.x == 0) {
        unsigned int* set = gate + 2 * (piece & 1u);
        const unsigned int t0 = cl_globaltimer_lo();
        unsigned int proposal = 1;
        while (cl_load_acquire(set) < blocks) {
            if (cl_load_acquire(set + 1) != 0 || cl_globaltimer_lo() - t0 > kClCheckInNs) {
                proposal = 2;
                break;
            }
            __nanosleep(64);
        }
        const unsigned int old = atomicCAS(set + 1, 0u, proposal);
        go = (old == 0 ? proposal : old) == 1;
        if (!go) atomicMin(gate + 4, piece);
        if (go && blockIdx.x == 0) {
            unsigned int* other = gate + 2 * ((piece + 1u) & 1u);
            other[0] = 0;
            other[1] = 0;
        }
    }
    return __syncthreads_or(go) != 0;
}

__device__ __noinline__ bool cl_count_in_call(unsigned int* gate, unsigned int piece)
{
    return cl_count_in(gate, piece);
}

__device__ __noinline__ bool cl_decide_call(unsigned int* gate, unsigned int blocks, unsigned int piece)
{
    return cl_decide(gate, blocks, piece);
}

// Waits until *f >= want; gives up after kClWaitNs of the GPU's global
// timer, records the failure in *err and returns false (the caller carries
// on with stale rows: the launch ends, its result is void, and the host
// reports the error).
__device__ __forceinline__ bool cl_wait_flag(const unsigned long long* f, unsigned long long want,
                                             unsigned int* err)
{
    const unsigned long long t0 = cl_globaltimer();
    while (cl_flag_acquire(f) < want) {
        // another wait of the launch gave up: its rows are void anyway
        if (*(volatile unsigned int*)err != 0) return false;
        if (cl_globaltimer() - t0 > kClWaitNs) {
            atomicExch(err, 1u);
            return false;
        }
        __nanosleep(100);
    }
    return true;
}

}  // namespace
}  // namespace ising

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

// Waits until *f >= want; gives up after kClWaitNs of the GPU's global
// timer, records the failure in *err and returns false (the caller carries
// on with stale rows: the launch ends, its result is void, and the host
// reports the error).
__device__ __forceinline__ bool cl_wait_flag(const unsigned long long* f, unsigned long long want,
                                             unsigned int* err)
{
    const unsigned long long t0 = cl_globaltimer();
    while (cl_flag_acquire(f) < want) {
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

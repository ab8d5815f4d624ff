// ising_sweep_record_noalloc: the record path for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a plug-in inside a host program that
// owns all device memory through its own pool, or a latency-critical loop in
// which an allocation (which may synchronise the device) is not acceptable.
// They hand in the packed lattice they already own and host arrays for the
// results; the only device memory this entry point touches besides those is
// the fixed array below, which lives in the library image and is created
// when the library is loaded on a device.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/ising.h"
#include "ising_internal.h"

namespace {

constexpr int kMaxRecords = ISING_NOALLOC_MAX_RECORDS;
constexpr int kSlots = ising::kCountSlots;
// Layout of the scratch array, in 64-bit words:
//   [0, kCounts)            count slots: record r, slot k -> 2 words (anti, up)
//   [kCounts, +kMaxRecords) E per record
//   [.., +kMaxRecords)      M per record
//   [kTOffset]              sweep counter the half-sweep kernel reads
constexpr size_t kCounts = (size_t)kMaxRecords * kSlots * 2;
constexpr size_t kEOffset = kCounts;
constexpr size_t kMOffset = kEOffset + kMaxRecords;
constexpr size_t kTOffset = kMOffset + kMaxRecords;
constexpr size_t kScratchWords = kTOffset + 32;   // the counter, padded to 256 bytes

// The scratch memory: every GPU that loads the library holds one copy
// (kScratchWords * 8 bytes, about 528 KB) until the process exits.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, so the address must come from the
// runtime; it is looked up on the first call on each device and cached.
int scratch_on_current_device(unsigned long long** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ising::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return ISING_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ising::cuda_fail(e, "cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ISING_OK;
}

__global__ void noalloc_set_sweep_kernel(unsigned long long* t, unsigned long long value)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t = value;
}

// E = 2 anti - 2 L^2 and M = 2 up - L^2 from the count slots of each record.
__global__ void noalloc_finalize_kernel(unsigned long long* scratch, int nrec, long long L)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const unsigned long long* slots = scratch + (size_t)r * kSlots * 2;
    unsigned long long anti = 0, up = 0;
    for (int k = 0; k < kSlots; ++k) {
        anti += slots[2 * k];
        up += slots[2 * k + 1];
    }
    const long long N = L * L;
    reinterpret_cast<long long*>(scratch + kEOffset)[r] = 2 * (long long)anti - 2 * N;
    reinterpret_cast<long long*>(scratch + kMOffset)[r] = 2 * (long long)up - N;
}

}  // namespace

extern "C" int ising_sweep_record_noalloc(uint64_t* dev_words0, uint64_t* dev_words1, int32_t L, uint64_t seed,
                                          double beta, uint64_t t0, int64_t n, int64_t every, int64_t* host_E,
                                          int64_t* host_M, void* stream)
{
    if (!dev_words0 || !dev_words1) return ISING_EINVAL;
    if (L < 4 || L > 32768 || (L % 2) != 0) return ISING_EINVAL;
    if (n < 0 || every < 1 || n > (int64_t)1 << 30) return ISING_EINVAL;
    if (std::isnan(beta) || beta < 0.0) return ISING_EINVAL;
    const int64_t nrec = n / every;
    if (nrec > kMaxRecords) return ISING_EINVAL;    // the fixed scratch holds kMaxRecords records

    unsigned long long* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != ISING_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // The array keeps the previous call's contents: clear the count slots.
    cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)(nrec > 0 ? nrec : 1) * kSlots * 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return ising::cuda_fail(e, "cudaMemsetAsync");
    noalloc_set_sweep_kernel<<<1, 1, 0, s>>>(scratch + kTOffset, t0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ising::cuda_fail(e, "noalloc_set_sweep_kernel");

    const ising::Geom g = ising::lattice_geom(L);
    uint64_t thr[2];
    ising::thresholds_for_beta(beta, thr);
    ising::SweepArgs a = ising::make_sweep_args(seed, thr, reinterpret_cast<const uint64_t*>(scratch + kTOffset));
    for (int64_t step = 1; step <= n; ++step) {
        a.t_off = (uint32_t)step;
        a.counts = nullptr;
        e = ising::launch_half_sweep(32, 4, 0, true, false, dev_words0, dev_words1, g, a, s);
        if (e != cudaSuccess) return ising::cuda_fail(e, "half_sweep colour 0");
        const bool rec = (step % every) == 0;
        if (rec) a.counts = scratch + (size_t)(step / every - 1) * kSlots * 2;
        e = ising::launch_half_sweep(32, 4, 1, true, rec, dev_words1, dev_words0, g, a, s);
        if (e != cudaSuccess) return ising::cuda_fail(e, "half_sweep colour 1");
    }
    if (nrec > 0) {
        noalloc_finalize_kernel<<<(unsigned)((nrec + 127) / 128), 128, 0, s>>>(scratch, (int)nrec, (long long)L);
        e = cudaGetLastError();
        if (e != cudaSuccess) return ising::cuda_fail(e, "noalloc_finalize_kernel");
        if (host_E) {
            e = cudaMemcpyAsync(host_E, scratch + kEOffset, (size_t)nrec * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return ising::cuda_fail(e, "cudaMemcpyAsync E");
        }
        if (host_M) {
            e = cudaMemcpyAsync(host_M, scratch + kMOffset, (size_t)nrec * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return ising::cuda_fail(e, "cudaMemcpyAsync M");
        }
    }
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ISING_OK : ising::cuda_fail(e, "cudaStreamSynchronize");
}

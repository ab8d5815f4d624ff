// Test helper: Philox4_32_10 blocks from cuRAND's device API, to pin the
// library's generator to NVIDIA's implementation of the published one.
// curand_init(seed, subsequence, offset): key = seed, the subsequence sets
// the high 64 bits of the counter and offset / 4 advances its low 64 bits;
// curand4() then returns the block of that counter.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_blocks_kernel(const unsigned int* ctr, unsigned int* out, int n, unsigned long long seed)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const unsigned long long lo = ((unsigned long long)ctr[4 * b + 1] << 32) | ctr[4 * b];
    const unsigned long long hi = ((unsigned long long)ctr[4 * b + 3] << 32) | ctr[4 * b + 2];
    curandStatePhilox4_32_10_t st;
    curand_init(seed, hi, 4ull * lo, &st);
    const uint4 v = curand4(&st);
    out[4 * b + 0] = v.x;
    out[4 * b + 1] = v.y;
    out[4 * b + 2] = v.z;
    out[4 * b + 3] = v.w;
}

extern "C" int curand_philox_blocks(unsigned long long seed, const unsigned int* host_ctr, unsigned int* host_out, int n)
{
    unsigned int* d = nullptr;
    if (cudaMalloc(&d, (size_t)n * 8 * sizeof(unsigned int)) != cudaSuccess) return 1;
    cudaMemcpy(d, host_ctr, (size_t)n * 4 * sizeof(unsigned int), cudaMemcpyHostToDevice);
    curand_blocks_kernel<<<(n + 127) / 128, 128>>>(d, d + 4 * n, n, seed);
    cudaError_t e = cudaMemcpy(host_out, d + 4 * n, (size_t)n * 4 * sizeof(unsigned int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e != cudaSuccess;
}

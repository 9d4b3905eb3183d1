// Test-only reference: cuRAND's device Philox4x32-10 (curand_Philox4x32_10 from curand_kernel.h)
// on caller-given (counter, key) tuples, built by the RNG test to check the library's own generator.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_philox(uint64_t n, const uint4* ctr, const uint2* key, uint4* out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// Host arrays: ctr u32[n][4], key u32[n][2], out u32[n][4].  Returns a cudaError_t value.
extern "C" int curand_philox_ref(uint64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 40 * n);
    if (e != cudaSuccess) return (int)e;
    uint4* dc = (uint4*)d;
    uint4* dout = dc + n;
    uint2* dk = (uint2*)(dout + n);
    e = cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_curand_philox<<<(unsigned)((n + 255) / 256), 256>>>(n, dc, dk, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return (int)e;
}

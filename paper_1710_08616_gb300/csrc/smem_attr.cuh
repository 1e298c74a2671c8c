// Dynamic shared-memory limits above 48 KB, set once per device: the kernel
// attribute belongs to the current device's context, so a process that drives
// several GPUs sets it on each of them.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace asuca {

template <typename K>
cudaError_t set_smem_once(K kernel, int bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

}  // namespace asuca

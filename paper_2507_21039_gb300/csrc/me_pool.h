// Temporary device buffers of the library (host-buffer staging, per-launch
// scratch) come from a private stream-ordered memory pool per device whose
// release threshold is unlimited: freed memory stays reserved for the next
// call instead of going back to the CUDA driver at every synchronisation, which the
// default pool (threshold 0) does, so that a repeated call maps no memory
// again.  The pool holds at most the largest set of buffers that were in
// flight at once; it lives until the process exits.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace me {

inline cudaMemPool_t staging_pool()
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t threshold = UINT64_MAX;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &threshold) != cudaSuccess) cudaGetLastError();
        pools[dev] = p;
    }
    return pools[dev];
}

// cudaMallocAsync from the staging pool (from the default pool if the private
// one could not be made, or while the stream is being captured into a graph,
// whose allocations the graph owns); free with cudaFreeAsync as usual
template <class T> cudaError_t staging_alloc(T** ptr, size_t bytes, cudaStream_t s)
{
    void** p = reinterpret_cast<void**>(ptr);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    cudaMemPool_t pool = cap == cudaStreamCaptureStatusNone ? staging_pool() : nullptr;
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

}  // namespace me

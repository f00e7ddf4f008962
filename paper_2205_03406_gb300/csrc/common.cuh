// Shared helpers of the hm CUDA library: error plumbing, device buffers,
// block reductions and a single-CTA scan for the small index arrays of the tree.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

// Status with a message; every internal function returns one.
struct Err {
    hm_status code = HM_OK;
    std::string msg;
    explicit operator bool() const { return code != HM_OK; }
};

inline Err ok() { return Err(); }
inline Err fail(hm_status c, const std::string &m) { Err e; e.code = c; e.msg = m; return e; }

#define HM_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return ::hm::fail(HM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

#define HM_LAUNCH(name)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess)                                                                \
            return ::hm::fail(HM_ECUDA, std::string("launch ") + name + ": " +                \
                                            cudaGetErrorString(e_));                          \
    } while (0)

#define HM_TRY(expr)                  \
    do {                              \
        ::hm::Err e__ = (expr);       \
        if (e__) return e__;          \
    } while (0)

// Stream on which the current API call allocates and frees (set on entry).
extern thread_local cudaStream_t g_alloc_stream;

// Sets g_alloc_stream for a scope (every entry point and worker thread).
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
    ~StreamScope() { g_alloc_stream = prev; }
    StreamScope(const StreamScope &) = delete;
    StreamScope &operator=(const StreamScope &) = delete;
};

// Kernel launches made by this library (every launch site calls this once).
void count_launch();
long long launches_so_far();

// Device allocations made by this library since it was loaded (every
// cudaMallocAsync of alloc() counts once).
void count_alloc();
long long allocs_so_far();

// Host-side fault injection for the error-path tests: with the environment
// variable HM_FAULT_ALLOC_AFTER=k set when the library is loaded, the device
// allocation after k successful ones fails once with HM_ENOMEM (before any
// CUDA call is made for it); unset, this is never true.
bool fault_alloc_now();

// A device allocation: move-only, freed (stream-ordered) when it goes out of
// scope, so temporaries of a call never outlive it and never force a device
// synchronisation.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void release() {
        if (p) cudaFreeAsync(p, g_alloc_stream);
        p = nullptr;
        bytes = 0;
    }
};

inline Err alloc(DBuf &b, size_t bytes) {
    b.release();
    if (bytes == 0) bytes = 16;
    if (fault_alloc_now()) return fail(HM_ENOMEM, "injected allocation failure (HM_FAULT_ALLOC_AFTER)");
    count_alloc();
    cudaError_t e = cudaMallocAsync(&b.p, bytes, g_alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(HM_ENOMEM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return ok();
}

// Grow-only reuse: keeps the allocation when it is already large enough.
inline Err ensure(DBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return ok();
    return alloc(b, bytes);
}

// Makes a context's device current for the duration of a call and restores
// the caller's device afterwards (nothing happens when no device is visible).
struct DeviceScope {
    int prev = -1, want = -1;
    explicit DeviceScope(int dev) : want(dev) {
        if (want < 0 || cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
            return;
        }
        if (prev != want) cudaSetDevice(want);
    }
    ~DeviceScope() {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};

// Opts a kernel into the largest dynamic shared memory the current device
// allows (its opt-in limit less the kernel's static shared memory) and checks
// that `need` bytes fit.  Every caller sets the same value, so jobs compressed
// concurrently on several host threads cannot lower each other's limit between
// one thread's setting and its launch.
template <class Kernel> inline Err allow_smem(Kernel *kernel, size_t need) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return fail(HM_ECUDA, "allow_smem: device attributes");
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)kernel) != cudaSuccess)
        return fail(HM_ECUDA, "allow_smem: kernel attributes");
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((int64_t)need > lim)
        return fail(HM_ENOTSUP, "kernel needs " + std::to_string(need) + " bytes of shared memory, the device allows " +
                                    std::to_string(lim));
    if (cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess)
        return fail(HM_ECUDA, "allow_smem: cudaFuncSetAttribute");
    return ok();
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

template <class T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread receives the result.  `sh` holds >= 32 T.
template <class T> __device__ __forceinline__ T block_sum(T v, T *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// Exclusive scan of n int64 values in place, by one CTA of 1024 threads
// (sizes here are at most a few million).  out[n] receives the total.
__global__ void k_scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n);

Err scan_exclusive(const int64_t *in_dev, int64_t *out_dev, int64_t n, cudaStream_t st);

// Convert int32 counts to int64 and exclusive-scan them: out has n+1 entries.
Err scan_counts_i32(const int *counts_dev, int64_t *out_dev, int64_t n, cudaStream_t st,
                    DBuf &tmp);

// Device-to-host reads into pageable memory drain the stream FIRST and copy
// after: a pageable copy queued behind a long kernel blocks inside the driver
// until that kernel ends, and holds up the pageable copies of every other host
// thread meanwhile (the colouring thread runs its kernels concurrently with
// the level loop).
template <class T> Err to_host(std::vector<T> &h, const void *d, size_t count, cudaStream_t st) {
    h.resize(count);
    HM_CUDA(cudaStreamSynchronize(st));
    if (count) {
        HM_CUDA(cudaMemcpyAsync(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    return ok();
}

template <class T> Err to_dev(DBuf &b, const std::vector<T> &h, cudaStream_t st) {
    HM_TRY(alloc(b, h.size() * sizeof(T)));
    if (!h.empty()) {
        HM_CUDA(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    }
    return ok();
}

template <class T> Err read_scalar(T &v, const void *d, cudaStream_t st) {
    HM_CUDA(cudaStreamSynchronize(st));
    HM_CUDA(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    return ok();
}

}  // namespace hm

// Device-side helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"

#define RS_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t rs_cuda_e_ = (call);                                                         \
        if (rs_cuda_e_ != cudaSuccess)                                                           \
            return rs::fail(RS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(rs_cuda_e_), \
                            __FILE__, __LINE__);                                                 \
    } while (0)

#define RS_LAUNCH_CHECK()                                                                        \
    do {                                                                                         \
        cudaError_t rs_cuda_e_ = cudaGetLastError();                                             \
        if (rs_cuda_e_ != cudaSuccess)                                                           \
            return rs::fail(RS_ECUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(rs_cuda_e_), \
                            __FILE__, __LINE__);                                                 \
    } while (0)

namespace rs {

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Raises the dynamic shared-memory limit of kernel `fn` on the current
// device to at least `bytes`.  The attribute belongs to a (function, device)
// pair, so the grant is remembered per pair and later calls with a size
// already granted cost one table lookup.
int smem_optin(const void *fn, size_t bytes);

// Device buffer owned by a handle.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int alloc(size_t n) {
        release();
        if (n == 0) return RS_OK;
        if (cudaMalloc(&p, n) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(RS_ENOMEM, "cudaMalloc(%zu) failed", n);
        }
        bytes = n;
        return RS_OK;
    }
    int upload(const void *src, size_t n) {
        RS_TRY(alloc(n));
        if (n && cudaMemcpy(p, src, n, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RS_ECUDA, "cudaMemcpy H2D failed");
        return RS_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return (T *)p; }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

}  // namespace rs

// Host-side helpers of device.h that keep state across calls.
#include <map>
#include <mutex>
#include <utility>

#include "device.h"

namespace rs {

int smem_optin(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> granted;
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &g = granted[{fn, dev}];
    if (g >= bytes) return RS_OK;
    RS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    g = bytes;
    return RS_OK;
}

}  // namespace rs

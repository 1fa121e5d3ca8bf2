// Allocation-free variant of the Cholesky orthonormalisation.
//
// rs_orthonormalize needs a device workspace that the caller allocates.
// Some callers cannot allocate device memory at the point where they need
// the operation: plugins handed pre-allocated buffers by a host framework
// that owns all device memory, or real-time loops that forbid cudaMalloc
// after start-up.  rs_orthonormalize_noalloc serves them: its scratch
// (overlap matrix, Cholesky factor, inverse and status word) lives in one
// file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.  The call is blocking (it reads
// the factorisation status back and synchronises its stream), so it is not
// for a stream under capture.
#include <mutex>

#include "device.h"
#include "linalg.h"

#ifndef RS_NOALLOC_MAX_STATES
#define RS_NOALLOC_MAX_STATES 256
#endif

namespace {

// Largest number of states the allocation-free call accepts.
constexpr int kMaxStates = RS_NOALLOC_MAX_STATES;
// S, U, U^-1, xi (n^2 each), n eigenvalues and the status words, for n = kMaxStates
constexpr size_t kScratchDoubles = 4 * (size_t)kMaxStates * kMaxStates + kMaxStates + 16;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch, looked up once per device (the host-side name
// is only a stand-in for the symbol, not a device address).
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

int scratch_address(void **out) {
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return rs::fail(RS_ECUDA, "rs_orthonormalize_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return rs::fail(RS_ECUDA, "rs_orthonormalize_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RS_OK;
}

}  // namespace

extern "C" int rs_orthonormalize_noalloc(const rs_grid *g, void *Psi_dev, int64_t ld, int nst, int dtype,
                                         void *stream) {
    if (!g || !Psi_dev) return rs::fail(RS_EINVAL, "rs_orthonormalize_noalloc: null argument");
    if (nst < 1 || ld < nst) return rs::fail(RS_EINVAL, "rs_orthonormalize_noalloc: bad nst or ld");
    if (nst > kMaxStates)
        return rs::fail(RS_EINVAL, "rs_orthonormalize_noalloc: nst = %d exceeds the fixed scratch limit of %d states",
                        nst, kMaxStates);
    if (dtype != RS_F64 && dtype != RS_F32) return rs::fail(RS_EINVAL, "rs_orthonormalize_noalloc: bad dtype");
    void *scratch = nullptr;
    RS_TRY(scratch_address(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    // every scratch word the call reads is written first by the call itself:
    // the overlap is zeroed before it is accumulated, the status word is always set
    RS_TRY(rs::orthonormalize_impl(g->npts, g->h * g->h * g->h, Psi_dev, ld, nst, dtype, scratch, st));
    RS_CUDA(cudaStreamSynchronize(st));  // the scratch is free again when the call returns
    return RS_OK;
}

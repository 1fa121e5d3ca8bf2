// Preconditioners of the block eigensolver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rsdft.h"

namespace rs {

class Precond {
   public:
    virtual ~Precond() = default;
    // W = K R for a block of nb residual columns; R [npts][ldr], W [npts][ldw].
    virtual int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
                      cudaStream_t st) = 0;
    virtual int set_weights(const float *w_dev, cudaStream_t st);
    virtual int kind() const = 0;   // RS_PRECOND_* (RS_PRECOND_CG for the CG iterations)
    static Precond *create(int kind, double filter_alpha, int64_t npts, int nb, int dtype);
    // n_iter CG iterations on the caller's shifted Hamiltonian (V = sigma, no projectors)
    static Precond *create_cg(rs_ham *shifted, int n_iter, int64_t npts, int nb, int dtype);
};

}  // namespace rs

// Internal accessors of the Hamiltonian handle shared with the solver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rsdft.h"

namespace rs {

int64_t ham_npts(const rs_ham *h);
double ham_dV(const rs_ham *h);
const int32_t *ham_map(const rs_ham *h);   // device point map [d0][d1][d2]
const int32_t *ham_loc(const rs_ham *h);   // device linear map index of every point
int ham_dim(const rs_ham *h, int axis);
// Device status word of the H psi kernel's bounded waits (nullptr when the
// handle has no such kernel): nonzero once a wait gave up.
int *ham_status_word(rs_ham *h);
struct DevBuf;
// Device scratch owned by h, grown to at least `bytes` (nullptr on failure).
DevBuf *ham_scratch(rs_ham *h, size_t bytes);

// W = K R with the face-neighbour smoothing filter
//   (K r)(p) = alpha r(p) + (1 - alpha)/6 sum_{6 face neighbours} r(n),
// r = 0 off the grid; R, W are [npts][ld] blocks of nb columns (dtype).
int ham_filter(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype, double alpha,
               cudaStream_t st);

}  // namespace rs

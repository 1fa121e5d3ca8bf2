// Learned preconditioner internals shared with the solver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rsdft.h"

namespace rs {

constexpr int LEARNED_WEIGHTS = 2160;   // [8][1][27] | [8][8][27] | [1][8][27]

// W = K R for nb FP32 residual columns; wq_dev: BF16-rounded weights (FP32
// storage); act: learned_act_floats(npts, nb) floats; dots: 128 doubles.
int learned_apply(const rs_ham *h, const float *R, int64_t ldr, float *W, int64_t ldw, int nb, const float *wq_dev,
                  float *act, double *dots, cudaStream_t st);
int64_t learned_act_floats(int64_t npts, int nb);
int learned_round_weights(const float *w, float *wq, cudaStream_t st);

}  // namespace rs

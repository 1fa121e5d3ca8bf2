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

// Training on tiles cut from (residual, target) column pairs (FP32
// [npts][ld], ncols columns), inputs and targets scaled by the residual's
// rms; w_dev holds the initial weights and receives the trained ones.
// Blocking.
int train_pairs_impl(const rs_ham *h, const rs_grid *g, const float *R_dev, const float *X_dev, int64_t ld, int ncols,
                     const rs_train_cfg &c, float *w_dev, float *loss_host, cudaStream_t st);

}  // namespace rs

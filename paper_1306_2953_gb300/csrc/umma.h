// Tensor-core (tcgen05) contractions of the FP32 mode (see umma.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rs {

// Workspace bytes for split operands of rows_a x K and rows_b x K.
int64_t umma_work_bytes(int64_t rows_a, int64_t rows_b, int64_t K);

// A caller-owned copy of the BF16x3 split of the X operand of umma_gram or
// umma_rowmul (each call keeps its own layout: buf must hold
// umma_split_cache_bytes of that call).  A call with a valid cache for the
// same X (pointer, columns, leading dimension, points) skips the split; the
// caller sets valid = false whenever X changes.
struct UmmaSplitCache {
    void *buf = nullptr;
    const float *src = nullptr;
    int n = 0;
    int64_t ld = 0, rows = 0;
    bool valid = false;
};
// bytes of the X split of umma_gram (gram = true; nx columns) or umma_rowmul
// (n columns) over npts points
int64_t umma_split_cache_bytes(bool gram, int64_t npts, int64_t ncols);

// S (nx x ny, FP64, row stride lds) = dV X^T Y, FP32 X [npts][ldx], Y [npts][ldy].
int umma_gram(const float *X, int64_t ldx, int nx, const float *Y, int64_t ldy, int ny, int64_t npts, double dV,
              double *S, int64_t lds, void *work, int *err, cudaStream_t st, UmmaSplitCache *xcache = nullptr);

// Y = alpha X C + beta Y; X FP32 [npts][ldx] (n columns), C FP64 [n][ldc]
// (m columns), Y FP32 [npts][ldy]; Y may alias X (X is split first; not
// with a cache, whose split would then be stale).
int umma_rowmul(const float *X, int64_t ldx, int n, const double *C, int64_t ldc, int m, float *Y, int64_t ldy,
                int64_t npts, double alpha, double beta, void *work, int *err, cudaStream_t st,
                UmmaSplitCache *xcache = nullptr);

}  // namespace rs

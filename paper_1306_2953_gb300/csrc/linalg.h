// Internal device linear-algebra entry points (see linalg.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rsdft.h"

namespace rs {

// S = dV X^T Y (nx x ny, FP64, row stride lds); X, Y are [npts][ld] of T.
// FP32 data: exact products with compensated accumulation, or (fast) plain
// FP32 accumulation within chunks of points combined in FP64.
template <typename T>
int gram(const T *X, int64_t ldx, int nx, const T *Y, int64_t ldy, int ny, int64_t npts, double dV, double *S,
         int64_t lds, cudaStream_t st, bool fast = false);

// Y = alpha X C + beta Y row by row; X [npts][ldx] (n columns), C FP64 [n][ldc]
// (m columns), Y [npts][ldy]; Y may alias X when beta == 0.
template <typename T>
int rowmul(const T *X, int64_t ldx, int n, const double *C, int64_t ldc, int m, T *Y, int64_t ldy, int64_t npts,
           double alpha, double beta, cudaStream_t st);

// out[k] = sum_p A[p][k] B[p][k] (FP64, exact products, compensated sum), k < ncols <= 256.
int coldots(int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, int ncols, int64_t npts, double *out,
            cudaStream_t st);

// Small dense FP64 helpers.
int gemm_small(int m, int n, int k, double alpha, const double *A, int lda, bool ta, const double *B, int ldb, bool tb,
               double beta, double *C, int ldc, cudaStream_t st);
int cholesky(double *A, int lda, int n, double rel, int *status_dev, cudaStream_t st);
int tri_inv(const double *U, int ldu, int n, double *X, int ldx, cudaStream_t st);
int symmetrize(double *A, int lda, int n, cudaStream_t st);

// Jacobi eigensolver in precision T on a copy of A (scratch: 2 n^2 T).
template <typename T>
int jacobi(const double *A, int lda, int n, int max_sweeps, double tol, double *w, double *V, int ldv, int *info,
           void *scratch, cudaStream_t st);

// Ogita-Aishima refinement of eigenvectors X of A; work: 4 n^2 + 1 doubles.
int refsyev(const double *A, int lda, double *X, int ldx, int n, double *lam, double *work, int iters,
            cudaStream_t st);

// Symmetric eigendecomposition A = V diag(w) V^T (ascending), FP64 result.
// refine > 0: FP32 Jacobi, `refine` Ogita-Aishima FP64 refinement steps and an
// FP64 Jacobi polish of V^T A V; refine = 0: FP64 Jacobi; refine < 0: FP32
// Jacobi only.  work: eigh_work_bytes(n).
size_t eigh_work_bytes(int n);
int eigh(const double *A, int lda, int n, double *w, double *V, int ldv, int refine, int *info_dev, void *work,
         cudaStream_t st);

// Layout of the workspace of orthonormalize / subspace_diag for n states.
struct LaWork {
    double *S, *U, *Ui, *xi, *eig;
    void *eigw;
    int *status;
    LaWork(void *base, int n) {
        double *d = reinterpret_cast<double *>(base);
        S = d;
        U = S + (size_t)n * n;
        Ui = U + (size_t)n * n;
        xi = Ui + (size_t)n * n;
        eig = xi + (size_t)n * n;
        status = reinterpret_cast<int *>(eig + n);
        eigw = reinterpret_cast<void *>(eig + n + 8);
    }
    static size_t bytes(int n) { return sizeof(double) * ((size_t)4 * n * n + n + 8) + eigh_work_bytes(n) + 256; }
};

// Tensor-core workspace for FP32 contractions (optional): base pointer,
// its size, and a device status word set when a tensor-core wait times out.
struct TcWork {
    void *p = nullptr;
    int64_t bytes = 0;
    int *err = nullptr;
    // inner iterations of the FP32 eigensolver: the full overlaps of Sec. VI
    // on the tensor cores as well, and the subspace eigenvectors from FP32
    // Jacobi alone (the closing FP64 Rayleigh-Ritz fixes the final accuracy)
    bool inner = false;
};

// Psi (n columns) <- Psi C in place (C FP64 n x n); FP32 data on the tensor
// cores when tc.p is set and large enough.
int rotate_inplace(void *Psi, int64_t ld, int n, const double *C, int64_t npts, int dtype, cudaStream_t st,
                   const TcWork &tc = TcWork());
// Psi <- Psi U^-1 with <Psi|Psi> = U^T U; w.Ui keeps U^-1.  Blocking; RS_ENOTSPD on failure.
int orthonormalize_impl(int64_t npts, double dV, void *Psi, int64_t ld, int n, int dtype, void *work, cudaStream_t st,
                        const TcWork &tc = TcWork());
// HPsi = H Psi, h = <Psi|H|Psi>, h xi = xi diag(eps), Psi <- Psi xi, HPsi <- HPsi xi; w.xi keeps xi.
int subspace_diag_impl(rs_ham *h, void *Psi, void *HPsi, int64_t ld, int n, int dtype, int nb, void *work,
                       double *eps_dev, cudaStream_t st, const TcWork &tc = TcWork());

}  // namespace rs
